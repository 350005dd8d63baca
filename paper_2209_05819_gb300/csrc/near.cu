// Near field of the HODLRdD product on the fly (Algorithm 2, leaf loop, and
// the IL blocks applied exactly): shared-memory tiles over box-relative FP32
// hi + lo coordinates for one or several right-hand sides, the final sum of
// the level contributions, and the direct O(N^2) comparator.
#include <algorithm>

#include "internal.cuh"
#include "pairs.cuh"

namespace hd {

namespace {

// Packed dense work (FP32, d <= 3, one right-hand side), one CTA per task.
// A task is up to kTileRows target rows [I0, I0 + m) of one box I at level l
// and a list of source ranges J. Coordinates are box-relative at level l and
// kept as FP32 pairs hi + lo (split from FP64 at build); a source is moved into
// I's frame by the exact FP32 offset (c_J - c_I) h_l with an error-free sum, so
// x_i - x_j = (hi_i - hi_j) + (lo_i - lo_j) keeps FP32 relative accuracy of the
// distance itself. Sources are staged through shared memory in chunks planned
// on the host (entry .z = position in the chunk, .w on a chunk's first entry =
// the entry after the chunk); then threads holding two target rows each sweep
// the chunk in S source stripes. Result: ynear[i] += scale * sum + diag * x_i
// (diag is passed as 0 except for the pass that owns the diagonal).
// HILO = false (option near_coords = 1): the hi parts alone, the lo parts are
// neither staged nor read.

// Barriers of the tile body: the whole CTA, or one 256-thread group of a
// larger CTA (named barrier `id`, the group's threads only).
struct SyncCta {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct SyncGroup {
  int id;
  __device__ __forceinline__ void operator()() const {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(kTileThreads) : "memory");
  }
};

// One task of the packed near field on kTileThreads threads (tid = the thread's
// index among them), staging through shi / slo (kTileCap entries each) and
// red / red2 (kTileThreads each); ends with a barrier, after which the staging
// arrays may be reused.
template <int D, int KID, bool HILO, class Sync>
__device__ __forceinline__ void tile_task(const int4 T, const int4* __restrict__ srcs,
                                          const float4* __restrict__ soff, const float4* __restrict__ Hi,
                                          const float4* __restrict__ Lo, const float* __restrict__ xt, float kc,
                                          float kscale, float kdiag, float* __restrict__ ynear, float4* shi,
                                          float4* slo, float* red, float* red2, int tid, Sync sync) {
  const int warp = tid >> 5, lane = tid & 31;
  // each thread holds two target rows, gi and gi + G with G = ceil(m / 2), and
  // sweeps one of S = 256 / G source stripes; the 256 - S G threads left over
  // sweep nothing (a power-of-two G would leave up to half the row slots empty
  // for boxes just above a power of two)
  const int G = max(1, (T.y + 1) / 2);
  const int S = kTileThreads / G;
  const int gi = tid % G, stripe = tid / G;
  const bool va = gi < T.y, vb = gi + G < T.y;
  const int ra = T.x + gi, rb = T.x + gi + G;
  float4 tha = make_float4(0.f, 0.f, 0.f, 0.f), tla = tha, thb = tha, tlb = tha;
  float xa = 0.f, xb = 0.f;
  if (va) {
    tha = Hi[ra];
    if (HILO) tla = Lo[ra];
    xa = xt[ra];
  }
  if (vb) {
    thb = Hi[rb];
    if (HILO) tlb = Lo[rb];
    xb = xt[rb];
  }
  float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
  for (int e = T.z; e < T.w;) {
    const int e1 = srcs[e].w;
    sync();  // the previous chunk has been consumed
    for (int b = e + warp; b < e1; b += kTileThreads / 32) {
      const int4 sj = srcs[b];
      const float4 of = soff[b];
      for (int k = lane; k < sj.y; k += 32) {
        const float4 h = Hi[sj.x + k];
        if (HILO) {
          const float4 l = Lo[sj.x + k];
          float ex, ey, ez;
          const float hx = two_sum(h.x, of.x, ex), hy = two_sum(h.y, of.y, ey), hz = two_sum(h.z, of.z, ez);
          shi[sj.z + k] = make_float4(hx, hy, hz, xt[sj.x + k]);
          slo[sj.z + k] = make_float4(l.x + ex, l.y + ey, l.z + ez, 0.f);
        } else {
          shi[sj.z + k] = make_float4(h.x + of.x, h.y + of.y, h.z + of.z, xt[sj.x + k]);
        }
      }
    }
    const int4 lastb = srcs[e1 - 1];
    const int n = lastb.z + lastb.y;
    sync();
    int f = stripe < S ? stripe : n;  // threads past the S stripes sweep nothing
#pragma unroll(HILO ? 1 : 2)
    for (; f + S < n; f += 2 * S) {
      const float4 h0 = shi[f], h1 = shi[f + S];
      if (HILO) {
        const float4 l0 = slo[f], l1 = slo[f + S];
        acc_pair<KID>(sqdist2<D>(tha, tla, h0, l0), kc, h0.w, a0);
        acc_pair<KID>(sqdist2<D>(thb, tlb, h0, l0), kc, h0.w, b0);
        acc_pair<KID>(sqdist2<D>(tha, tla, h1, l1), kc, h1.w, a1);
        acc_pair<KID>(sqdist2<D>(thb, tlb, h1, l1), kc, h1.w, b1);
      } else {
        acc_pair<KID>(sqdist1<D>(tha, h0), kc, h0.w, a0);
        acc_pair<KID>(sqdist1<D>(thb, h0), kc, h0.w, b0);
        acc_pair<KID>(sqdist1<D>(tha, h1), kc, h1.w, a1);
        acc_pair<KID>(sqdist1<D>(thb, h1), kc, h1.w, b1);
      }
    }
    if (f < n) {
      const float4 h0 = shi[f];
      if (HILO) {
        const float4 l0 = slo[f];
        acc_pair<KID>(sqdist2<D>(tha, tla, h0, l0), kc, h0.w, a0);
        acc_pair<KID>(sqdist2<D>(thb, tlb, h0, l0), kc, h0.w, b0);
      } else {
        acc_pair<KID>(sqdist1<D>(tha, h0), kc, h0.w, a0);
        acc_pair<KID>(sqdist1<D>(thb, h0), kc, h0.w, b0);
      }
    }
    e = e1;
  }
  red[tid] = a0 + a1;
  red2[tid] = b0 + b1;
  sync();
  if (stripe == 0) {
    float acc_a = 0.f, acc_b = 0.f;
    for (int s = 0; s < S; ++s) {
      acc_a += red[s * G + gi];
      acc_b += red2[s * G + gi];
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const bool v = q == 0 ? va : vb;
      if (!v) continue;
      const int row = q == 0 ? ra : rb;
      const float acc = q == 0 ? acc_a : acc_b;
      ynear[row] += kscale * acc + kdiag * (q == 0 ? xa : xb);
    }
  }
  sync();  // red and the staging arrays are reused by the next task
}

template <int D, int KID, bool HILO>
__global__ void __launch_bounds__(kTileThreads, 3) k_tile(const int4* __restrict__ tasks, int64_t t0, int64_t t1,
                                                      const int4* __restrict__ srcs, const float4* __restrict__ soff,
                                                      const float4* __restrict__ Hi, const float4* __restrict__ Lo,
                                                      const float* __restrict__ xt, float kc, float kscale,
                                                      float kdiag, float* __restrict__ ynear) {
  __shared__ float4 shi[kTileCap];  // hi coordinates in the task's frame, x_j in .w
  __shared__ float4 slo[kTileCap];  // lo coordinates
  __shared__ float red[kTileThreads], red2[kTileThreads];
  for (int64_t it = t0 + blockIdx.x; it < t1; it += gridDim.x)
    tile_task<D, KID, HILO>(tasks[it], srcs, soff, Hi, Lo, xt, kc, kscale, kdiag, ynear, shi, slo, red, red2,
                            (int)threadIdx.x, SyncCta{});
}

// The same passes on a fixed set of SMs (option near_sms): one CTA per SM of
// kSplitGroups groups of kTileThreads threads, launched with a whole SM's
// shared memory so that no other CTA shares its SM. All passes are one launch:
// a group takes the next task from a counter (tasks of all passes numbered in
// pass order) and adds its sums into its pass's own buffer, so passes never
// write the same row at the same time; the final sum adds the buffers in pass
// order.
template <int D, int KID, bool HILO>
__global__ void __launch_bounds__(kSplitGroups* kTileThreads, 1)
    k_tile_split(const __grid_constant__ SplitArgs a, const int4* __restrict__ tasks, const int4* __restrict__ srcs,
                 const float4* __restrict__ soff, const float* __restrict__ xt, float kc) {
  extern __shared__ __align__(16) unsigned char split_sm[];
  const int g = (int)threadIdx.x / kTileThreads, tid = (int)threadIdx.x % kTileThreads;
  float4* shi = reinterpret_cast<float4*>(split_sm + (size_t)g * kSplitGroupBytes);
  float4* slo = shi + kTileCap;
  float* red = reinterpret_cast<float*>(slo + kTileCap);
  float* red2 = red + kTileThreads;
  int* slot = reinterpret_cast<int*>(red2 + kTileThreads);
  const SyncGroup sync{1 + g};
  for (;;) {
    if (tid == 0) *slot = atomicAdd(a.ctr, 1);
    sync();
    int64_t k = *slot;
    if (k >= a.total) break;  // every thread of the group read the same value
    int p = 0;
    while (p + 1 < a.npass && k >= a.pass[p].n) k -= a.pass[p++].n;
    const SplitPass& P = a.pass[p];
    tile_task<D, KID, HILO>(tasks[P.t0 + k], srcs, soff, P.Hi, P.Lo, xt, kc, P.scale, P.diag, P.out, shi, slo, red,
                            red2, tid, sync);
  }
}

// Direct on-the-fly product y = K x over all N^2 pairs (FP32 arithmetic, d <=
// 3, one right-hand side): the exact-by-definition comparator of the HODLRdD
// product. Coordinates relative to the bounding cube's corner as FP32 hi + lo
// pairs; each CTA holds 2 x kDirectThreads targets and streams every source
// through shared memory; sums are compensated.
constexpr int kDirectThreads = 128;

template <int D, int KID>
__global__ void __launch_bounds__(kDirectThreads) k_direct(const float4* __restrict__ Hi,
                                                          const float4* __restrict__ Lo,
                                                          const float* __restrict__ xt, int64_t N, float kc,
                                                          float kscale, float kdiag,
                                                          const int32_t* __restrict__ perm, float* __restrict__ y) {
  __shared__ float4 shi[kTileCap];
  __shared__ float4 slo[kTileCap];
  const int tid = threadIdx.x;
  const int64_t ra = (int64_t)blockIdx.x * 2 * kDirectThreads + tid, rb = ra + kDirectThreads;
  float4 tha = make_float4(0.f, 0.f, 0.f, 0.f), tla = tha, thb = tha, tlb = tha;
  if (ra < N) {
    tha = Hi[ra];
    tla = Lo[ra];
  }
  if (rb < N) {
    thb = Hi[rb];
    tlb = Lo[rb];
  }
  // compensated (Kahan) sums: N terms per target
  float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f, ca0 = 0.f, ca1 = 0.f, cb0 = 0.f, cb1 = 0.f;
  auto kadd = [](float& sum, float& comp, float term) {
    const float yv = term - comp;
    const float t = sum + yv;
    comp = (t - sum) - yv;
    sum = t;
  };
  for (int64_t c0 = 0; c0 < N; c0 += kTileCap) {
    const int n = N - c0 < kTileCap ? (int)(N - c0) : kTileCap;
    __syncthreads();  // the previous chunk has been consumed
    for (int k = tid; k < n; k += kDirectThreads) {
      float4 h = Hi[c0 + k];
      h.w = xt[c0 + k];
      shi[k] = h;
      slo[k] = Lo[c0 + k];
    }
    __syncthreads();
    int f = 0;
    for (; f + 1 < n; f += 2) {
      const float4 h0 = shi[f], l0 = slo[f], h1 = shi[f + 1], l1 = slo[f + 1];
      kadd(a0, ca0, f32k<KID>(sqdist2<D>(tha, tla, h0, l0), kc) * h0.w);
      kadd(b0, cb0, f32k<KID>(sqdist2<D>(thb, tlb, h0, l0), kc) * h0.w);
      kadd(a1, ca1, f32k<KID>(sqdist2<D>(tha, tla, h1, l1), kc) * h1.w);
      kadd(b1, cb1, f32k<KID>(sqdist2<D>(thb, tlb, h1, l1), kc) * h1.w);
    }
    if (f < n) {
      const float4 h0 = shi[f], l0 = slo[f];
      kadd(a0, ca0, f32k<KID>(sqdist2<D>(tha, tla, h0, l0), kc) * h0.w);
      kadd(b0, cb0, f32k<KID>(sqdist2<D>(thb, tlb, h0, l0), kc) * h0.w);
    }
  }
  a0 -= ca0;
  a1 -= ca1;
  b0 -= cb0;
  b1 -= cb1;
  if (ra < N) y[perm[ra]] = kscale * (a0 + a1) + kdiag * xt[ra];
  if (rb < N) y[perm[rb]] = kscale * (b0 + b1) + kdiag * xt[rb];
}

// Box-relative coordinates at level l as FP32 pairs: x - (lo + c_box h) = hi + lo
// (the difference formed in FP64).
__global__ void k_relhilo(const double* __restrict__ p64, int64_t N, int d, int l, const int32_t* __restrict__ bstart,
                          const uint64_t* __restrict__ bkey, int64_t nb, const double* __restrict__ lo, double h,
                          float4* __restrict__ Hi, float4* __restrict__ Lo) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t a = 0, b = nb;  // last box with bstart <= i
    while (b - a > 1) {
      const int64_t mid = (a + b) >> 1;
      if (bstart[mid] <= i) a = mid; else b = mid;
    }
    const uint64_t key = bkey[a];
    float hv[4] = {0.f, 0.f, 0.f, 0.f}, lv[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < d && k < 4; ++k) {
      int64_t c = 0;
      for (int bit = 0; bit < l; ++bit) c |= (int64_t)((key >> (d * bit + k)) & 1u) << bit;
      const double v = p64[(int64_t)k * N + i] - (lo[k] + (double)c * h);
      hv[k] = __double2float_rn(v);
      lv[k] = __double2float_rn(v - (double)hv[k]);
    }
    Hi[i] = make_float4(hv[0], hv[1], hv[2], hv[3]);
    Lo[i] = make_float4(lv[0], lv[1], lv[2], lv[3]);
  }
}

// y[perm[i] * ldy + c0 + r] = near(i, r) + sum over the level slices of
// y_l(i, r) (one per level, two with the mixed storage's FP16 tail), for NR
// right-hand sides stored NR per point.
template <int NR>
__global__ void k_finish(const float* __restrict__ ynear, int nnear, const float* __restrict__ ylev, int slices,
                         int64_t N, const int32_t* __restrict__ perm, float* __restrict__ y, int ldy, int c0) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    float tot[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) tot[r] = ynear[i * NR + r];
    for (int p = 1; p < nnear; ++p)  // near-field passes summed into buffers of their own
#pragma unroll
      for (int r = 0; r < NR; ++r) tot[r] += ynear[((int64_t)p * N + i) * NR + r];
    for (int l = 0; l < slices; ++l)
#pragma unroll
      for (int r = 0; r < NR; ++r) tot[r] += ylev[((int64_t)l * N + i) * NR + r];
    float* out = y + (int64_t)perm[i] * ldy + c0;
#pragma unroll
    for (int r = 0; r < NR; ++r) out[r] = tot[r];
  }
}

// Packed dense work for NR right-hand sides (FP32 arithmetic, d <= 4), one CTA
// per task as in k_tile, two target rows per thread, specialised on the kernel
// function: each pair's kernel value multiplies the NR values of its source. x_t and ynear hold NR values per
// point. Dynamic shared memory: kTileCap staged sources (hi, lo, NR values)
// and the stripe reduction.
// The stripe reduction (kTileThreads x 2 x NR floats) reuses the staging area.
template <int NR>
constexpr size_t tile_nr_smem() {
  const size_t stage = (size_t)kTileCap * (2 * sizeof(float4) + NR * sizeof(float));
  const size_t red = (size_t)kTileThreads * 2 * NR * sizeof(float);
  return stage > red ? stage : red;
}

template <int NR>
__device__ __forceinline__ void load_x(const float* p, float (&v)[NR]) {
  if constexpr (NR % 4 == 0) {
#pragma unroll
    for (int r = 0; r < NR; r += 4) {
      const float4 q = *reinterpret_cast<const float4*>(p + r);
      v[r] = q.x; v[r + 1] = q.y; v[r + 2] = q.z; v[r + 3] = q.w;
    }
  } else if constexpr (NR == 2) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    v[0] = q.x; v[1] = q.y;
  } else {
#pragma unroll
    for (int r = 0; r < NR; ++r) v[r] = p[r];
  }
}

template <int D, int NR, int KID>
__global__ void __launch_bounds__(kTileThreads, 2) k_tile_nr(const int4* __restrict__ tasks, int64_t t0, int64_t t1,
                                                         const int4* __restrict__ srcs,
                                                         const float4* __restrict__ soff,
                                                         const float4* __restrict__ Hi, const float4* __restrict__ Lo,
                                                         const float* __restrict__ xt, float kc, float kscale,
                                                         float kdiag, float* __restrict__ ynear, int ldx, int cx) {
  extern __shared__ __align__(16) char tsm[];
  float4* shi = reinterpret_cast<float4*>(tsm);
  float4* slo = shi + kTileCap;
  float* sx = reinterpret_cast<float*>(slo + kTileCap);
  float* red = reinterpret_cast<float*>(tsm);  // kTileThreads * 2 * NR, after the last chunk
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int64_t it = t0 + blockIdx.x; it < t1; it += gridDim.x) {
    const int4 T = tasks[it];
    // each thread holds two target rows, gi and gi + G
    int lg = 0;
    while ((2 << lg) < T.y) ++lg;
    const int G = 1 << lg, S = kTileThreads >> lg;
    const int gi = tid & (G - 1), stripe = tid >> lg;
    const bool va = gi < T.y, vb = gi + G < T.y;
    const int ra = T.x + gi, rb = ra + G;
    float4 tha = make_float4(0.f, 0.f, 0.f, 0.f), tla = tha, thb = tha, tlb = tha;
    if (va) {
      tha = Hi[ra];
      tla = Lo[ra];
    }
    if (vb) {
      thb = Hi[rb];
      tlb = Lo[rb];
    }
    float aa[NR], ab[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) aa[r] = ab[r] = 0.f;
    for (int e = T.z; e < T.w;) {
      const int e1 = srcs[e].w;
      __syncthreads();  // the previous chunk has been consumed
      for (int b = e + warp; b < e1; b += kTileThreads / 32) {
        const int4 sj = srcs[b];
        const float4 of = soff[b];
        for (int k = lane; k < sj.y; k += 32) {
          const float4 h = Hi[sj.x + k], l = Lo[sj.x + k];
          float ex, ey, ez, ew;
          const float hx = two_sum(h.x, of.x, ex), hy = two_sum(h.y, of.y, ey), hz = two_sum(h.z, of.z, ez),
                      hw = two_sum(h.w, of.w, ew);
          shi[sj.z + k] = make_float4(hx, hy, hz, hw);
          slo[sj.z + k] = make_float4(l.x + ex, l.y + ey, l.z + ez, l.w + ew);
          float xv[NR];
          load_x<NR>(xt + (int64_t)(sj.x + k) * ldx + cx, xv);
#pragma unroll
          for (int r = 0; r < NR; ++r) sx[(sj.z + k) * NR + r] = xv[r];
        }
      }
      const int4 lastb = srcs[e1 - 1];
      const int n = lastb.z + lastb.y;
      __syncthreads();
#pragma unroll 2
      for (int f = stripe; f < n; f += S) {
        const float4 hs = shi[f], ls = slo[f];
        const float ka = f32k<KID>(sqdist2<D>(tha, tla, hs, ls), kc);
        const float kb = f32k<KID>(sqdist2<D>(thb, tlb, hs, ls), kc);
        float xv[NR];
        load_x<NR>(sx + f * NR, xv);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          aa[r] = fmaf(ka, xv[r], aa[r]);
          ab[r] = fmaf(kb, xv[r], ab[r]);
        }
      }
      e = e1;
    }
    __syncthreads();  // every thread is done with the staged sources
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      red[(2 * tid) * NR + r] = aa[r];
      red[(2 * tid + 1) * NR + r] = ab[r];
    }
    __syncthreads();
    if (stripe == 0) {
      for (int q = 0; q < 2; ++q) {
        const bool v = q == 0 ? va : vb;
        if (!v) continue;
        const int row = q == 0 ? ra : rb;
        for (int r = 0; r < NR; ++r) {
          float sum = 0.f;
          for (int s2 = 0; s2 < S; ++s2) sum += red[(2 * (s2 * G + gi) + q) * NR + r];
          ynear[(int64_t)row * ldx + cx + r] += kscale * sum + kdiag * xt[(int64_t)row * ldx + cx + r];
        }
      }
    }
    __syncthreads();  // red and the staging arrays are reused by the next task
  }
}


template <int D, int KID, bool HILO>
void launch_tiles_kc(hodlrdd_s* h, cudaStream_t st, const float* xt) {
  const Plan& P = h->plan;
  const float kc = (float)kernel_const(h->K);
  const float ks = (float)h->K.scale, kd = (float)h->K.diag;
  float* yn = h->ynear.p;
  // one CTA per task (the hardware scheduler balances tasks of unequal size)
  auto grid = [&](int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(n, INT32_MAX)); };
  for (const DenseLevel& DL : P.coarse4) {
    k_tile<D, KID, HILO><<<grid(DL.t1 - DL.t0), kTileThreads, 0, st>>>(P.tasks4.p, DL.t0, DL.t1, P.srcs4.p, P.soff4.p,
                                                                P.hi4[DL.level].p, P.lo4[DL.level].p, xt, kc, ks,
                                                                0.f, yn);
    h->launches += 1;
  }
  if (P.excl4.t1 > P.excl4.t0) {
    // low-rank leaf blocks that the parent tiles also evaluate: subtract them
    k_tile<D, KID, HILO><<<grid(P.excl4.t1 - P.excl4.t0), kTileThreads, 0, st>>>(
        P.tasks4.p, P.excl4.t0, P.excl4.t1, P.srcs4.p, P.soff4.p, P.hi4[P.excl4.level].p, P.lo4[P.excl4.level].p, xt,
        kc, -ks, 0.f, yn);
    h->launches += 1;
  }
  k_tile<D, KID, HILO><<<grid(P.leaf4.t1 - P.leaf4.t0), kTileThreads, 0, st>>>(
      P.tasks4.p, P.leaf4.t0, P.leaf4.t1, P.srcs4.p, P.soff4.p, P.hi4[P.leaf4.level].p, P.lo4[P.leaf4.level].p, xt,
      kc, ks, kd, yn);
  h->launches += 1;
}

template <int D, int KID>
void launch_tiles_k(hodlrdd_s* h, cudaStream_t st, const float* xt) {
  if (h->opt.near_coords == 1) launch_tiles_kc<D, KID, false>(h, st, xt);
  else launch_tiles_kc<D, KID, true>(h, st, xt);
}

// The passes of launch_tiles_kc as one k_tile_split launch on near_sms CTAs,
// pass p summing into ynear + p N (zeroed here with the task counter).
template <int D, int KID, bool HILO>
int launch_split_kc(hodlrdd_s* h, cudaStream_t st, const float* xt) {
  static PerDeviceOnce attr;
  HD_TRY(attr.run([] {
    int dev = 0, optin = 0;
    HD_CUDA(cudaGetDevice(&dev));
    HD_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    HD_CUDA(cudaFuncSetAttribute(k_tile_split<D, KID, HILO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - 512));
    return (int)HODLRDD_OK;
  }));
  const Plan& P = h->plan;
  SplitArgs a{};
  int np = 0;
  auto add = [&](int64_t t0, int64_t t1, int level, float scale, float diag) {
    if (t1 <= t0) return;
    a.pass[np] = SplitPass{t0, t1 - t0, P.hi4[level].p, P.lo4[level].p, scale, diag, h->ynear.p + (size_t)np * h->N};
    a.total += t1 - t0;
    ++np;
  };
  const float ks = (float)h->K.scale, kd = (float)h->K.diag;
  for (const DenseLevel& DL : P.coarse4) add(DL.t0, DL.t1, DL.level, ks, 0.f);
  add(P.excl4.t0, P.excl4.t1, P.excl4.level, -ks, 0.f);
  add(P.leaf4.t0, P.leaf4.t1, P.leaf4.level, ks, kd);
  a.npass = np;
  a.ctr = h->nctr.p;
  HD_CUDA(cudaMemsetAsync(h->ynear.p, 0, (size_t)np * h->N * sizeof(float), st));
  HD_CUDA(cudaMemsetAsync(h->nctr.p, 0, sizeof(int32_t), st));
  int dev = 0, optin = 0;
  HD_CUDA(cudaGetDevice(&dev));
  HD_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // the per-block limit less 512 bytes: less than the 1 KB a CTA reserves stays free on the SM
  k_tile_split<D, KID, HILO><<<h->opt.near_sms, kSplitGroups * kTileThreads, optin - 512, st>>>(
      a, P.tasks4.p, P.srcs4.p, P.soff4.p, xt, (float)kernel_const(h->K));
  h->launches += 1;
  HD_CUDA(cudaGetLastError());
  return HODLRDD_OK;
}

template <int D, int KID>
int launch_split_k(hodlrdd_s* h, cudaStream_t st, const float* xt) {
  return h->opt.near_coords == 1 ? launch_split_kc<D, KID, false>(h, st, xt) : launch_split_kc<D, KID, true>(h, st, xt);
}

template <int D>
int launch_split_d(hodlrdd_s* h, cudaStream_t st, const float* xt) {
  switch (h->K.id) {
    case HODLRDD_K_LOG: return launch_split_k<D, HODLRDD_K_LOG>(h, st, xt);
    case HODLRDD_K_INV_R: return launch_split_k<D, HODLRDD_K_INV_R>(h, st, xt);
    case HODLRDD_K_MATERN32: return launch_split_k<D, HODLRDD_K_MATERN32>(h, st, xt);
    case HODLRDD_K_GAUSS: return launch_split_k<D, HODLRDD_K_GAUSS>(h, st, xt);
    case HODLRDD_K_EXP: return launch_split_k<D, HODLRDD_K_EXP>(h, st, xt);
    case HODLRDD_K_INV_R2_4D: return launch_split_k<D, HODLRDD_K_INV_R2_4D>(h, st, xt);
    case HODLRDD_K_R: return launch_split_k<D, HODLRDD_K_R>(h, st, xt);
    case HODLRDD_K_SIN: return launch_split_k<D, HODLRDD_K_SIN>(h, st, xt);
    default: return launch_split_k<D, HODLRDD_K_INV_SQRT1P>(h, st, xt);
  }
}

template <int D>
void launch_tiles_d(hodlrdd_s* h, cudaStream_t st, const float* xt) {
  switch (h->K.id) {
    case HODLRDD_K_LOG: launch_tiles_k<D, HODLRDD_K_LOG>(h, st, xt); break;
    case HODLRDD_K_INV_R: launch_tiles_k<D, HODLRDD_K_INV_R>(h, st, xt); break;
    case HODLRDD_K_MATERN32: launch_tiles_k<D, HODLRDD_K_MATERN32>(h, st, xt); break;
    case HODLRDD_K_GAUSS: launch_tiles_k<D, HODLRDD_K_GAUSS>(h, st, xt); break;
    case HODLRDD_K_EXP: launch_tiles_k<D, HODLRDD_K_EXP>(h, st, xt); break;
    case HODLRDD_K_INV_R2_4D: launch_tiles_k<D, HODLRDD_K_INV_R2_4D>(h, st, xt); break;
    case HODLRDD_K_R: launch_tiles_k<D, HODLRDD_K_R>(h, st, xt); break;
    case HODLRDD_K_SIN: launch_tiles_k<D, HODLRDD_K_SIN>(h, st, xt); break;
    default: launch_tiles_k<D, HODLRDD_K_INV_SQRT1P>(h, st, xt); break;
  }
}

}  // namespace

int split_passes(const hodlrdd_s* h) {
  const Plan& P = h->plan;
  int np = 0;
  for (const DenseLevel& DL : P.coarse4) np += DL.t1 > DL.t0;
  np += P.excl4.t1 > P.excl4.t0;
  np += P.leaf4.t1 > P.leaf4.t0;
  return np;
}

int launch_tiles_split(hodlrdd_s* h, cudaStream_t st, const float* xt) {
  switch (h->d) {
    case 1: return launch_split_d<1>(h, st, xt);
    case 2: return launch_split_d<2>(h, st, xt);
    default: return launch_split_d<3>(h, st, xt);
  }
}

// Packed near-field launches (FP32, d <= 3, one right-hand side) on stream st,
// accumulating into ynear (zeroed here).
void launch_tiles(hodlrdd_s* h, cudaStream_t st, const float* xt) {
  cudaMemsetAsync(h->ynear.p, 0, (size_t)h->N * sizeof(float), st);
  switch (h->d) {
    case 1: launch_tiles_d<1>(h, st, xt); break;
    case 2: launch_tiles_d<2>(h, st, xt); break;
    default: launch_tiles_d<3>(h, st, xt); break;
  }
}


namespace {
template <int D, int NR, int KID>
int launch_tiles_nr_dnk(hodlrdd_s* h, cudaStream_t st, const float* xt, int ldx, int cx) {
  static PerDeviceOnce attr;
  HD_TRY(attr.run([] {
    HD_CUDA(cudaFuncSetAttribute(k_tile_nr<D, NR, KID>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tile_nr_smem<NR>()));
    return (int)HODLRDD_OK;
  }));
  const Plan& P = h->plan;
  const float kc = (float)kernel_const(h->K);
  const float ks = (float)h->K.scale, kd = (float)h->K.diag;
  float* yn = h->ynear.p;
  const size_t smem = tile_nr_smem<NR>();
  auto grid = [&](int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(n, INT32_MAX)); };
  for (const DenseLevel& DL : P.coarse4) {
    k_tile_nr<D, NR, KID><<<grid(DL.t1 - DL.t0), kTileThreads, smem, st>>>(
        P.tasks4.p, DL.t0, DL.t1, P.srcs4.p, P.soff4.p, P.hi4[DL.level].p, P.lo4[DL.level].p, xt, kc, ks, 0.f, yn, ldx, cx);
    h->launches += 1;
  }
  if (P.excl4.t1 > P.excl4.t0) {
    k_tile_nr<D, NR, KID><<<grid(P.excl4.t1 - P.excl4.t0), kTileThreads, smem, st>>>(
        P.tasks4.p, P.excl4.t0, P.excl4.t1, P.srcs4.p, P.soff4.p, P.hi4[P.excl4.level].p, P.lo4[P.excl4.level].p, xt,
        kc, -ks, 0.f, yn, ldx, cx);
    h->launches += 1;
  }
  k_tile_nr<D, NR, KID><<<grid(P.leaf4.t1 - P.leaf4.t0), kTileThreads, smem, st>>>(
      P.tasks4.p, P.leaf4.t0, P.leaf4.t1, P.srcs4.p, P.soff4.p, P.hi4[P.leaf4.level].p, P.lo4[P.leaf4.level].p, xt,
      kc, ks, kd, yn, ldx, cx);
  h->launches += 1;
  return HODLRDD_OK;
}

template <int D, int NR>
int launch_tiles_nr_dn(hodlrdd_s* h, cudaStream_t st, const float* xt, int ldx, int cx) {
  switch (h->K.id) {
    case HODLRDD_K_LOG: return launch_tiles_nr_dnk<D, NR, HODLRDD_K_LOG>(h, st, xt, ldx, cx);
    case HODLRDD_K_INV_R: return launch_tiles_nr_dnk<D, NR, HODLRDD_K_INV_R>(h, st, xt, ldx, cx);
    case HODLRDD_K_MATERN32: return launch_tiles_nr_dnk<D, NR, HODLRDD_K_MATERN32>(h, st, xt, ldx, cx);
    case HODLRDD_K_GAUSS: return launch_tiles_nr_dnk<D, NR, HODLRDD_K_GAUSS>(h, st, xt, ldx, cx);
    case HODLRDD_K_EXP: return launch_tiles_nr_dnk<D, NR, HODLRDD_K_EXP>(h, st, xt, ldx, cx);
    case HODLRDD_K_INV_R2_4D: return launch_tiles_nr_dnk<D, NR, HODLRDD_K_INV_R2_4D>(h, st, xt, ldx, cx);
    case HODLRDD_K_R: return launch_tiles_nr_dnk<D, NR, HODLRDD_K_R>(h, st, xt, ldx, cx);
    case HODLRDD_K_SIN: return launch_tiles_nr_dnk<D, NR, HODLRDD_K_SIN>(h, st, xt, ldx, cx);
    default: return launch_tiles_nr_dnk<D, NR, HODLRDD_K_INV_SQRT1P>(h, st, xt, ldx, cx);
  }
}

template <int D>
int launch_tiles_nr_d(hodlrdd_s* h, cudaStream_t st, const float* xt, int nr, int ldx, int cx) {
  switch (nr) {
    case 1: return launch_tiles_nr_dn<D, 1>(h, st, xt, ldx, cx);
    case 2: return launch_tiles_nr_dn<D, 2>(h, st, xt, ldx, cx);
    case 4: return launch_tiles_nr_dn<D, 4>(h, st, xt, ldx, cx);
    case 8: return launch_tiles_nr_dn<D, 8>(h, st, xt, ldx, cx);
    default: return launch_tiles_nr_dn<D, 16>(h, st, xt, ldx, cx);
  }
}

__global__ void k_gather1(const float* __restrict__ x, const int32_t* __restrict__ perm, int64_t N,
                          float* __restrict__ xt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    xt[i] = x[perm[i]];
}
}  // namespace

// Packed near field for nr in {1, 2, 4, 8, 16} right-hand sides (FP32
// arithmetic, d <= 4) on stream st. x_t and ynear hold ldx values per point
// (ldx = 0: nr), of which columns cx .. cx + nr - 1 are applied. With ldx = 0
// ynear is zeroed here; otherwise the caller zeroes it and the columns add in.
int launch_tiles_nr(hodlrdd_s* h, cudaStream_t st, const float* xt, int nr, int ldx, int cx) {
  if (ldx == 0) {
    ldx = nr;
    cx = 0;
    HD_CUDA(cudaMemsetAsync(h->ynear.p, 0, (size_t)h->N * nr * sizeof(float), st));
  }
  switch (h->d) {
    case 1: HD_TRY(launch_tiles_nr_d<1>(h, st, xt, nr, ldx, cx)); break;
    case 2: HD_TRY(launch_tiles_nr_d<2>(h, st, xt, nr, ldx, cx)); break;
    case 3: HD_TRY(launch_tiles_nr_d<3>(h, st, xt, nr, ldx, cx)); break;
    default: HD_TRY(launch_tiles_nr_d<4>(h, st, xt, nr, ldx, cx)); break;
  }
  HD_CUDA(cudaGetLastError());
  return HODLRDD_OK;
}

// y = near + sum of the level slices, scattered to the original order.
int launch_finish(hodlrdd_s* h, cudaStream_t st, const float* ylev, int slices, float* y, int nr, int ldy, int c0,
                  int nnear) {
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  const int grid = (int)std::min<int64_t>((h->N + 255) / 256, sms * 16);
  const float* yn = h->ynear.p;
  switch (nr) {
    case 1: k_finish<1><<<grid, 256, 0, st>>>(yn, nnear, ylev, slices, h->N, h->perm.p, y, ldy, c0); break;
    case 2: k_finish<2><<<grid, 256, 0, st>>>(yn, nnear, ylev, slices, h->N, h->perm.p, y, ldy, c0); break;
    case 4: k_finish<4><<<grid, 256, 0, st>>>(yn, nnear, ylev, slices, h->N, h->perm.p, y, ldy, c0); break;
    case 8: k_finish<8><<<grid, 256, 0, st>>>(yn, nnear, ylev, slices, h->N, h->perm.p, y, ldy, c0); break;
    default: k_finish<16><<<grid, 256, 0, st>>>(yn, nnear, ylev, slices, h->N, h->perm.p, y, ldy, c0); break;
  }
  h->launches += 1;
  HD_CUDA(cudaGetLastError());
  return HODLRDD_OK;
}

// Box-relative hi + lo coordinates of every point at level l.
int launch_relhilo(hodlrdd_s* h, int l, float4* Hi, float4* Lo, const double* dlo, cudaStream_t st) {
  const Level& L = h->lv[l];
  k_relhilo<<<(int)std::min<int64_t>((h->N + 255) / 256, 152 * 16), 256, 0, st>>>(
      h->pts64.p, h->N, h->d, l, L.bstart.p, L.bkey.p, L.nb, dlo, h->plan.h_box[l], Hi, Lo);
  HD_CUDA(cudaGetLastError());
  return HODLRDD_OK;
}

namespace {
template <int D>
void launch_direct_d(hodlrdd_s* h, cudaStream_t st, const float* xt, float* y) {
  const Plan& P = h->plan;
  const float kc = (float)kernel_const(h->K);
  const float ks = (float)h->K.scale, kd = (float)h->K.diag;
  const int grid = (int)((h->N + 2 * kDirectThreads - 1) / (2 * kDirectThreads));
  const float4* Hi = P.hi4[0].p;
  const float4* Lo = P.lo4[0].p;
  switch (h->K.id) {
#define HD_DIRECT(K) \
  case K: k_direct<D, K><<<grid, kDirectThreads, 0, st>>>(Hi, Lo, xt, h->N, kc, ks, kd, h->perm.p, y); break;
    HD_DIRECT(HODLRDD_K_LOG) HD_DIRECT(HODLRDD_K_INV_R) HD_DIRECT(HODLRDD_K_MATERN32) HD_DIRECT(HODLRDD_K_GAUSS)
    HD_DIRECT(HODLRDD_K_EXP) HD_DIRECT(HODLRDD_K_INV_R2_4D) HD_DIRECT(HODLRDD_K_R) HD_DIRECT(HODLRDD_K_SIN)
    default: k_direct<D, HODLRDD_K_INV_SQRT1P><<<grid, kDirectThreads, 0, st>>>(Hi, Lo, xt, h->N, kc, ks, kd,
                                                                                h->perm.p, y);
#undef HD_DIRECT
  }
}
}  // namespace

int launch_direct(hodlrdd_s* h, const float* x, float* y, cudaStream_t st) {
  if (h->opt.precision == HODLRDD_PREC_FP64 || h->d > 3) {
    set_error("hodlrdd_direct: needs an FP32, FP16 or BF16 handle and d <= 3");
    return HODLRDD_ERR_UNSUPPORTED;
  }
  Plan& P = h->plan;
  if (P.hi4.empty()) P.hi4.resize(h->kappa + 1);
  if (P.lo4.empty()) P.lo4.resize(h->kappa + 1);
  if (!P.hi4[0].p) {  // cube-relative coordinates, made on the first call
    std::vector<double> hlo(h->lo, h->lo + h->d);
    DevBuf<double> dlo;
    HD_TRY(upload(dlo, hlo, st));
    HD_TRY(P.hi4[0].alloc(h->N));
    HD_TRY(P.lo4[0].alloc(h->N));
    const Level& L = h->lv[0];
    HD_TRY(launch_relhilo(h, 0, P.hi4[0].p, P.lo4[0].p, dlo.p, st));
    HD_CUDA(cudaStreamSynchronize(st));
  }
  float* xt = reinterpret_cast<float*>(h->xt.p) + (size_t)kGuard;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  k_gather1<<<(int)std::min<int64_t>((h->N + 255) / 256, sms * 16), 256, 0, st>>>(x, h->perm.p, h->N, xt);
  switch (h->d) {
    case 1: launch_direct_d<1>(h, st, xt, y); break;
    case 2: launch_direct_d<2>(h, st, xt, y); break;
    default: launch_direct_d<3>(h, st, xt, y); break;
  }
  HD_CUDA(cudaGetLastError());
  h->launches += 2;
  return HODLRDD_OK;
}


}  // namespace hd
