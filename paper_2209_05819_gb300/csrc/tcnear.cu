// Near field of the FP16X2 (tensor-core) form for a chunk of 64 right-hand
// sides (Algorithm 2, leaf loop, and the IL blocks applied exactly): every
// kernel value K(i, j) of a task is evaluated once, on the CUDA cores, from the
// box-relative FP32 hi + lo coordinates (as in the other near-field kernels),
// and the 64-wide accumulation Y(I) += K(I, S) X(S) runs on the tensor cores.
//
// Per task (target rows [I0, I0 + m) and a list of source ranges) and 128-row
// tile: the sources are taken in chunks of 64; for each chunk the CTA writes
//   A = K(tile rows, chunk)  as FP16 hi + 2^-11 lo planes (MN-major: one
//       128-byte row per source holds 64 targets, 128-byte swizzle),
//   B = X(chunk, 64) / sigma_x  split the same way,
// and one thread issues the hi.hi, hi.lo and lo.hi MMAs (lo the plain residual
// v - hi) into one tensor-memory accumulator per chunk. The tensor cores
// truncate when they add into an accumulator; started afresh every chunk (four
// MMA steps), each chunk's sum keeps that error to a few 2^-24 of itself, and
// the chunk sums are added with round-to-nearest FP32 additions into a running
// total in tensor memory (two chunks behind, so the adds overlap the MMAs).
// Chunks are double-buffered: the next chunk's kernel values are computed while
// the tensor cores consume the previous one. The kernels taken here are bounded
// on any point set in FP32 range (exp-type, r, sin, log r, 1/sqrt(1 + r): |K|
// <= 745 at most), so the FP16 high part never overflows, and a small value's
// subnormal low part still leaves an absolute error of 2^-25 of the largest
// entry; the singular power laws (1/r, 1/r^2) use the FP32 tiles.
#include <algorithm>

#include "internal.cuh"
#include "pairs.cuh"
#include "tcgen05.cuh"

namespace hd {
namespace {

constexpr int kNrThreads = 256;
constexpr int kNrKC = 64;                       // sources per chunk
constexpr int kNrPlane = kNrKC * 128;           // one plane: 64 rows x 128 bytes
constexpr int kNrStageBytes = 6 * kNrPlane;     // A (hi, lo) x (half 0, 1) + B (hi, lo)
constexpr int kNrSmem = 2 * kNrStageBytes + 1024;
constexpr int kNrEntWin = 256;                  // source entries whose prefix sums are held at once
constexpr int kNrTmemCols = 256;                // chunk accumulators D0, D1 and the tile total

static_assert(kNrSmem <= 110 * 1024, "two near-field CTAs per SM");

// First entry e of [0, n) with pre[e + 1] > k (pre ascending, pre[0] = 0).
__device__ __forceinline__ int find_entry(const int* pre, int n, int k) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= k) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ uint32_t pack2(__half a, __half b) {
  return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

// v = hi + lo with hi = fp16(v) and lo = fp16(v - hi): the plain residual,
// so that all three products land in one accumulator.
__device__ __forceinline__ void split_plain(float v, __half& hi, __half& lo) {
  hi = __float2half_rn(v);
  lo = __float2half_rn(v - __half2float(hi));
}

// Adds accumulator `src` into the running total `tot` (or copies it, first),
// 64 columns of this warp's 32 lanes, with round-to-nearest FP32 additions.
__device__ __forceinline__ void tmem_accumulate(uint32_t src, uint32_t tot, bool first) {
#pragma unroll
  for (int c0 = 0; c0 < kTcR; c0 += 16) {
    float a[16], b[16];
    tmem_ld16(src + c0, a);
    if (!first) tmem_ld16(tot + c0, b);
    tmem_wait_ld();
    if (!first)
#pragma unroll
      for (int i = 0; i < 16; ++i) a[i] += b[i];
    tmem_st16(tot + c0, a);
  }
  tmem_wait_st();
}

template <int D, int KID>
__global__ void __launch_bounds__(kNrThreads, 2) k_tc_near(const int4* __restrict__ tasks, int64_t t0, int64_t t1,
                                                            const int4* __restrict__ srcs,
                                                            const float4* __restrict__ soff,
                                                            const float4* __restrict__ Hi,
                                                            const float4* __restrict__ Lo,
                                                            const float* __restrict__ xt,
                                                            const unsigned int* __restrict__ colmax, float kc,
                                                            float kscale, float kdiag, float* __restrict__ ynear,
                                                            const int2* __restrict__ tbase,
                                                            const float2* __restrict__ tsd,
                                                            TcPack pk, int32_t* __restrict__ err) {
  const int2* __restrict__ tbox = pk.tbox;
  const int32_t* __restrict__ brow = pk.brow;
  const float4* __restrict__ boff = pk.boff;
  const uint32_t* __restrict__ emask = pk.emask;
  extern __shared__ __align__(1024) unsigned char nr_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(nr_raw) + 1023) & ~uintptr_t(1023));
  __shared__ float4 s_hi[2][kNrKC], s_lo[2][kNrKC];
  __shared__ int s_row[2][kNrKC];
  __shared__ uint32_t s_mask[2][kNrKC];  // boxes of the task that read the source
  __shared__ int s_brow[32];             // packed task: first row of each box
  __shared__ float4 s_boff[32];          // packed task: each box's offset into the task's frame
  __shared__ int s_pre[kNrEntWin + 1];
  __shared__ float s_sx[kTcR], s_isx[kTcR];
  __shared__ __align__(8) uint64_t mma_done[2], dready, fin;
  __shared__ uint32_t tmem_base;
  __shared__ int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid < kTcR) {
    s_sx[tid] = pow2_above(__uint_as_float(colmax[tid]));
    s_isx[tid] = 1.f / s_sx[tid];  // a power of two: exact
  }
  if (tid == 0) {
    bar_init(&mma_done[0], 1);
    bar_init(&mma_done[1], 1);
    bar_init(&dready, 1);
    bar_init(&fin, 1);
    s_ok = 1;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                 "r"(kNrTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // tensor memory: chunk accumulators D0, D1 (by chunk parity) and the tile's total
  const uint32_t tmem = tmem_base;
  const uint32_t lanebase = (uint32_t)((warp & 3) * 32) << 16;
  const uint32_t d_tot = tmem + 128 + lanebase;
  const int bq = (tid & 3) * 16;                        // B: this thread's 16 columns
  const int ac = tid & 15, ahh = ac >> 3, acc8 = ac & 7;  // A: 8 consecutive tile rows
  // kernels smooth in r^2 (Matern-3/2, Gaussian) lose nothing from the FP32
  // rounding of box-relative coordinates (an absolute error of r^2 of 2^-24
  // of the box size squared moves K by as much): the low parts are not read
  constexpr bool kSmooth = KID == HODLRDD_K_MATERN32 || KID == HODLRDD_K_GAUSS;
  int64_t g = 0;   // chunks issued by this CTA (stage g & 1)
  int64_t mt = 0;  // tiles with products (dready parity)
  bool ok = true;

  for (int64_t it = t0 + blockIdx.x; it < t1 && ok; it += gridDim.x) {
    const int4 T = tasks[it];
    // forest launches: the task's coordinate and point bases, scale and diagonal
    const int2 base = tbase ? tbase[it] : make_int2(0, 0);
    const float2 sd = tsd ? tsd[it] : make_float2(kscale, kdiag);
    const float4* __restrict__ Ht = Hi + base.x;
    const float4* __restrict__ Lt = Lo + base.x;
    const float* __restrict__ xb = xt + (int64_t)base.y * kTcR;
    float* __restrict__ yb = ynear + (int64_t)base.y * kTcR;
    // packed tasks: several small boxes, each with its first row and frame offset
    const int2 tb = tbox ? tbox[it] : make_int2(0, 1);
    if (tid < tb.y) {
      s_brow[tid] = tbox ? brow[tb.x + tid] : 0;
      s_boff[tid] = tbox ? boff[tb.x + tid] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    for (int r0 = 0; r0 < T.y && ok; r0 += 128) {
      const int mm = min(128, T.y - r0);
      // the thread's 8 targets (rows r0 + 8 ac + i of the task), moved into the
      // task's frame, and the box each belongs to (5 bits per row)
      float4 th[8], tl[8];
      bool tv[8];
      uint64_t bidx = 0;
      int bi = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = 8 * ac + i;
        tv[i] = r < mm;
        while (bi + 1 < tb.y && s_brow[bi + 1] <= r0 + r) ++bi;
        bidx |= (uint64_t)bi << (5 * i);
        const float4 ph = tv[i] ? Ht[T.x + r0 + r] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 pl = tv[i] && !kSmooth ? Lt[T.x + r0 + r] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 of = s_boff[bi];
        float ex, ey, ez, ew;
        th[i] = make_float4(two_sum(ph.x, of.x, ex), two_sum(ph.y, of.y, ey), two_sum(ph.z, of.z, ez),
                            two_sum(ph.w, of.w, ew));
        tl[i] = make_float4(pl.x + ex, pl.y + ey, pl.z + ez, pl.w + ew);
      }
      int c = 0;  // chunks of this tile; chunk c accumulates into D(c & 1), added into the total two chunks later
      for (int w0 = T.z; w0 < T.w && ok; w0 += kNrEntWin) {
        const int nw = min(kNrEntWin, T.w - w0);
        __syncthreads();  // s_pre of the previous window is no longer read
        if (warp == 0) {
          // prefix sums of the window's entry sizes (one warp, 32 at a time)
          int carry = 0;
          if (lane == 0) s_pre[0] = 0;
          for (int b = 0; b < nw; b += 32) {
            int v = b + lane < nw ? srcs[w0 + b + lane].y : 0;
            for (int o = 1; o < 32; o <<= 1) {
              const int u = __shfl_up_sync(0xffffffffu, v, o);
              if (lane >= o) v += u;
            }
            if (b + lane < nw) s_pre[b + lane + 1] = carry + v;
            carry += __shfl_sync(0xffffffffu, v, 31);
          }
        }
        __syncthreads();
        const int nsrc = s_pre[nw];
        for (int k0 = 0; k0 < nsrc; k0 += kNrKC, ++g, ++c) {
          const int st = (int)(g & 1);
          unsigned char* stage = sm + st * kNrStageBytes;
          if (g >= 2) {
            // the MMAs of two chunks ago are done: their stage is free, their accumulator final
            if (tid == 0) s_ok = bar_wait(&mma_done[st], (uint32_t)(((g >> 1) - 1) & 1), err, 10) ? 1 : 0;
            __syncthreads();
            if (!s_ok) {
              ok = false;
              break;
            }
          }
          if (c >= 2 && warp < 4) {
            tc_fence_after();
            tmem_accumulate(tmem + (uint32_t)((c & 1) * 64) + lanebase, d_tot, c == 2);
          }
          // the chunk's sources, moved into the target box's frame
          if (tid < kNrKC) {
            const int k = k0 + tid;
            int row = -1;
            uint32_t msk = 0u;
            float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
            if (k < nsrc) {
              const int e = find_entry(s_pre, nw, k);
              const int4 sj = srcs[w0 + e];
              const float4 of = soff[w0 + e];
              msk = emask ? emask[w0 + e] : ~0u;
              row = sj.x + (k - s_pre[e]);
              const float4 ph = Ht[row], pl = Lt[row];
              float ex, ey, ez, ew;
              h = make_float4(two_sum(ph.x, of.x, ex), two_sum(ph.y, of.y, ey), two_sum(ph.z, of.z, ez),
                              two_sum(ph.w, of.w, ew));
              l = make_float4(pl.x + ex, pl.y + ey, pl.z + ez, pl.w + ew);
            }
            s_hi[st][tid] = h;
            s_lo[st][tid] = l;
            s_row[st][tid] = row;
            s_mask[st][tid] = msk;
          }
          __syncthreads();
          // B: source row k = tid / 4, columns bq .. bq + 15, scaled by 1 / sigma_x, as hi and lo planes
          {
            const int k = tid >> 2;
            const int row = s_row[st][k];
            unsigned char* bh = stage + 4 * kNrPlane;
            unsigned char* bl = bh + kNrPlane;
#pragma unroll
            for (int half8 = 0; half8 < 2; ++half8) {
              const int n0 = bq + 8 * half8;
              float v[8];
              if (row >= 0) {
                const float4 a = *reinterpret_cast<const float4*>(xb + (int64_t)row * kTcR + n0);
                const float4 b = *reinterpret_cast<const float4*>(xb + (int64_t)row * kTcR + n0 + 4);
                v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
              } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) v[i] = 0.f;
              }
              __half hh[8], ll[8];
#pragma unroll
              for (int i = 0; i < 8; ++i) split_plain(v[i] * s_isx[n0 + i], hh[i], ll[i]);
              const int phys = k * 128 + (((n0 >> 3) ^ (k & 7)) << 4);
              *reinterpret_cast<uint4*>(bh + phys) =
                  make_uint4(pack2(hh[0], hh[1]), pack2(hh[2], hh[3]), pack2(hh[4], hh[5]), pack2(hh[6], hh[7]));
              *reinterpret_cast<uint4*>(bl + phys) =
                  make_uint4(pack2(ll[0], ll[1]), pack2(ll[2], ll[3]), pack2(ll[4], ll[5]), pack2(ll[6], ll[7]));
            }
          }
          // A: kernel values of the thread's 8 targets with sources tid / 16 + 16 j
#pragma unroll 1
          for (int j = 0; j < 4; ++j) {
            const int k = (tid >> 4) + 16 * j;
            const bool sv = s_row[st][k] >= 0;
            const uint32_t msk = s_mask[st][k];
            const float4 sh = s_hi[st][k], sl = s_lo[st][k];
            __half hh[8], ll[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              float f = 0.f;
              const bool reads = (msk >> (uint32_t)((bidx >> (5 * i)) & 31u)) & 1u;
              if (tv[i] && sv && reads)
                f = f32k<KID>(kSmooth ? sqdist1<D>(th[i], sh) : sqdist2<D>(th[i], tl[i], sh, sl), kc);
              split_plain(f, hh[i], ll[i]);
            }
            const int phys = k * 128 + ((acc8 ^ (k & 7)) << 4);
            *reinterpret_cast<uint4*>(stage + ahh * kNrPlane + phys) =
                make_uint4(pack2(hh[0], hh[1]), pack2(hh[2], hh[3]), pack2(hh[4], hh[5]), pack2(hh[6], hh[7]));
            *reinterpret_cast<uint4*>(stage + (2 + ahh) * kNrPlane + phys) =
                make_uint4(pack2(ll[0], ll[1]), pack2(ll[2], ll[3]), pack2(ll[4], ll[5]), pack2(ll[6], ll[7]));
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
          tc_fence_before();
          __syncthreads();
          if (tid == 0) {
            tc_fence_after();
            const uint32_t base = saddr(stage);
            const uint32_t dc = tmem + (uint32_t)((c & 1) * 64);
            const int ksteps = (min(kNrKC, nsrc - k0) + 15) / 16;
            for (int ks = 0; ks < ksteps; ++ks) {
              const uint32_t off = (uint32_t)ks * 2048u;
              const uint64_t ah = smem_desc(base + off, kNrPlane, 1024);
              const uint64_t al = smem_desc(base + 2 * kNrPlane + off, kNrPlane, 1024);
              const uint64_t bh = smem_desc(base + 4 * kNrPlane + off, kNrPlane, 1024);
              const uint64_t bl = smem_desc(base + 5 * kNrPlane + off, kNrPlane, 1024);
              mma_f16(dc, ah, bh, ks > 0 ? 1u : 0u);
              mma_f16(dc, ah, bl, 1u);
              mma_f16(dc, al, bh, 1u);
            }
            mma_commit(&mma_done[st]);
          }
        }
      }
      if (!ok) break;
      if (c > 0) {
        // the tile's last MMAs are done: add the chunks not yet in the total
        if (tid == 0) {
          mma_commit(&dready);
          s_ok = bar_wait(&dready, (uint32_t)(mt & 1), err, 11) ? 1 : 0;
        }
        __syncthreads();
        ++mt;
        if (!s_ok) {
          ok = false;
          break;
        }
        if (warp < 4) {
          tc_fence_after();
          for (int cc = c >= 2 ? c - 2 : 0; cc < c; ++cc)
            tmem_accumulate(tmem + (uint32_t)((cc & 1) * 64) + lanebase, d_tot, cc == 0);
        }
      }
      // y(row) += kscale sigma_x total + kdiag x(row)
      if (warp < 4) {
        const int r = warp * 32 + lane;
        const int64_t row = (int64_t)T.x + r0 + r;
#pragma unroll
        for (int c0 = 0; c0 < kTcR; c0 += 16) {
          float v[16];
          if (c > 0) {
            tmem_ld16(d_tot + c0, v);
            tmem_wait_ld();
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = 0.f;
          }
          if (r < mm) {
            float* yp = yb + row * kTcR + c0;
            const float* xp = xb + row * kTcR + c0;
#pragma unroll
            for (int i = 0; i < 16; i += 4) {
              const float4 x4 = *reinterpret_cast<const float4*>(xp + i);
              float4 y4 = *reinterpret_cast<const float4*>(yp + i);
              y4.x += sd.x * s_sx[c0 + i] * v[i] + sd.y * x4.x;
              y4.y += sd.x * s_sx[c0 + i + 1] * v[i + 1] + sd.y * x4.y;
              y4.z += sd.x * s_sx[c0 + i + 2] * v[i + 2] + sd.y * x4.z;
              y4.w += sd.x * s_sx[c0 + i + 3] * v[i + 3] + sd.y * x4.w;
              *reinterpret_cast<float4*>(yp + i) = y4;
            }
          }
        }
      }
      tc_fence_before();
      __syncthreads();  // the accumulators are free for the next tile
    }
  }
  // every MMA of this CTA has completed before its tensor memory is freed
  if (tid == 0 && g > 0) {
    mma_commit(&fin);
    bar_wait(&fin, 0, err, 12);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kNrTmemCols) : "memory");
  }
}

}  // namespace
}  // namespace hd

namespace hd {
namespace {

template <int D, int KID>
int tc_near_dk(hodlrdd_s* h, cudaStream_t st, const float* xt, const unsigned int* colmax) {
  static PerDeviceOnce attr;
  HD_TRY(attr.run([] {
    HD_CUDA(cudaFuncSetAttribute(k_tc_near<D, KID>, cudaFuncAttributeMaxDynamicSharedMemorySize, kNrSmem));
    return (int)HODLRDD_OK;
  }));
  const Plan& P = h->plan;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  const float kc = (float)kernel_const(h->K);
  const float ks = (float)h->K.scale, kd = (float)h->K.diag;
  auto run = [&](const DenseLevel& DL, float scale, float diag) {
    const int64_t n = DL.t1 - DL.t0;
    if (n <= 0) return;
    // one CTA per task (tasks sorted by decreasing work): the block scheduler
    // balances the SMs dynamically
    const int grid = (int)std::min<int64_t>(n, INT32_MAX);
    k_tc_near<D, KID><<<grid, kNrThreads, kNrSmem, st>>>(P.tasks4.p, DL.t0, DL.t1, P.srcs4.p, P.soff4.p,
                                                          P.hi4[DL.level].p, P.lo4[DL.level].p, xt, colmax, kc, scale,
                                                          diag, h->ynear.p, nullptr, nullptr, tc_pack(P), h->err.p);
    h->launches += 1;
  };
  for (const DenseLevel& DL : P.coarse4) run(DL, ks, 0.f);
  if (P.excl4.t1 > P.excl4.t0) run(P.excl4, -ks, 0.f);  // low-rank leaf blocks the parent tiles also cover
  run(P.leaf4, ks, kd);
  HD_CUDA(cudaGetLastError());
  return HODLRDD_OK;
}

template <int D>
int tc_near_d(hodlrdd_s* h, cudaStream_t st, const float* xt, const unsigned int* colmax) {
  switch (h->K.id) {
    case HODLRDD_K_LOG: return tc_near_dk<D, HODLRDD_K_LOG>(h, st, xt, colmax);
    case HODLRDD_K_MATERN32: return tc_near_dk<D, HODLRDD_K_MATERN32>(h, st, xt, colmax);
    case HODLRDD_K_GAUSS: return tc_near_dk<D, HODLRDD_K_GAUSS>(h, st, xt, colmax);
    case HODLRDD_K_EXP: return tc_near_dk<D, HODLRDD_K_EXP>(h, st, xt, colmax);
    case HODLRDD_K_R: return tc_near_dk<D, HODLRDD_K_R>(h, st, xt, colmax);
    case HODLRDD_K_SIN: return tc_near_dk<D, HODLRDD_K_SIN>(h, st, xt, colmax);
    default: return tc_near_dk<D, HODLRDD_K_INV_SQRT1P>(h, st, xt, colmax);
  }
}

}  // namespace

bool tc_near_supported(const hodlrdd_s* h) {
  return h->d <= 4 && tc_near_kernel(h->K.id) && h->plan.tasks4.n > 0;
}

// The near field of one chunk of kTcR right-hand sides on the tensor cores,
// accumulated into ynear (which the caller zeroes).
int launch_tc_near(hodlrdd_s* h, cudaStream_t st, const float* xt, const unsigned int* colmax) {
  switch (h->d) {
    case 1: return tc_near_d<1>(h, st, xt, colmax);
    case 2: return tc_near_d<2>(h, st, xt, colmax);
    case 3: return tc_near_d<3>(h, st, xt, colmax);
    default: return tc_near_d<4>(h, st, xt, colmax);
  }
}

}  // namespace hd

namespace hd {
namespace {

template <int D, int KID>
int tc_near_raw_dk(cudaStream_t st, int64_t ntask, const int4* tasks, const int4* srcs, const float4* soff,
                   const float4* Hi, const float4* Lo, const float* xt, const unsigned int* colmax, float kc,
                   float* ynear, const int2* tbase, const float2* tsd, TcPack pk, int32_t* err) {
  static PerDeviceOnce attr;
  HD_TRY(attr.run([] {
    HD_CUDA(cudaFuncSetAttribute(k_tc_near<D, KID>, cudaFuncAttributeMaxDynamicSharedMemorySize, kNrSmem));
    return (int)HODLRDD_OK;
  }));
  if (ntask <= 0) return HODLRDD_OK;
  k_tc_near<D, KID><<<(int)std::min<int64_t>(ntask, INT32_MAX), kNrThreads, kNrSmem, st>>>(
      tasks, 0, ntask, srcs, soff, Hi, Lo, xt, colmax, kc, 1.f, 0.f, ynear, tbase, tsd, pk, err);
  HD_CUDA(cudaGetLastError());
  return HODLRDD_OK;
}

template <int D>
int tc_near_raw_d(int kid, cudaStream_t st, int64_t ntask, const int4* tasks, const int4* srcs, const float4* soff,
                  const float4* Hi, const float4* Lo, const float* xt, const unsigned int* colmax, float kc,
                  float* ynear, const int2* tbase, const float2* tsd, TcPack pk, int32_t* err) {
#define HD_NEAR_RAW(K) \
  tc_near_raw_dk<D, K>(st, ntask, tasks, srcs, soff, Hi, Lo, xt, colmax, kc, ynear, tbase, tsd, pk, err)
  switch (kid) {
    case HODLRDD_K_LOG: return HD_NEAR_RAW(HODLRDD_K_LOG);
    case HODLRDD_K_MATERN32: return HD_NEAR_RAW(HODLRDD_K_MATERN32);
    case HODLRDD_K_GAUSS: return HD_NEAR_RAW(HODLRDD_K_GAUSS);
    case HODLRDD_K_EXP: return HD_NEAR_RAW(HODLRDD_K_EXP);
    case HODLRDD_K_R: return HD_NEAR_RAW(HODLRDD_K_R);
    case HODLRDD_K_SIN: return HD_NEAR_RAW(HODLRDD_K_SIN);
    default: return HD_NEAR_RAW(HODLRDD_K_INV_SQRT1P);
  }
#undef HD_NEAR_RAW
}

}  // namespace

// One launch of the tensor-core near field over tasks whose coordinate and
// point bases, scale and diagonal come per task (tasks of several trees).
int launch_tc_near_raw(int d, int kid, cudaStream_t st, int64_t ntask, const int4* tasks, const int4* srcs,
                       const float4* soff, const float4* Hi, const float4* Lo, const float* xt,
                       const unsigned int* colmax, float kc, float* ynear, const int2* tbase, const float2* tsd,
                       TcPack pk, int32_t* err) {
  switch (d) {
    case 1: return tc_near_raw_d<1>(kid, st, ntask, tasks, srcs, soff, Hi, Lo, xt, colmax, kc, ynear, tbase, tsd, pk, err);
    case 2: return tc_near_raw_d<2>(kid, st, ntask, tasks, srcs, soff, Hi, Lo, xt, colmax, kc, ynear, tbase, tsd, pk, err);
    case 3: return tc_near_raw_d<3>(kid, st, ntask, tasks, srcs, soff, Hi, Lo, xt, colmax, kc, ynear, tbase, tsd, pk, err);
    default: return tc_near_raw_d<4>(kid, st, ntask, tasks, srcs, soff, Hi, Lo, xt, colmax, kc, ynear, tbase, tsd, pk, err);
  }
}

}  // namespace hd
