// The low-rank applies of Algorithm 2 on the tensor cores (precision FP16X2),
// for chunks of up to 64 right-hand sides:
//
//   V-apply  t(J-block columns) = V_J^T X(J)      per source box J and 128 columns
//   U-apply  y_l(I)             = U_I  T(I)       per target box I and 128 rows
//
// Both are D (128 x 64, FP32, in tensor memory) = A (128 x K) B (K x 64) with A
// a factor panel (MN-major: 64 consecutive M entries per 128-byte row, K rows)
// and B rows of an FP32 array (x_t or t), split on the fly into FP16 pieces.
// Every value v is carried as hi = fp16(v / s) and lo = fp16((v / s - hi) 2^11)
// with s a power of two; the products hi.hi go to one accumulator and hi.lo +
// lo.hi to a second, and the epilogue forms s_A s_B (D_hi + 2^-11 D_lo). The
// scaled low part stays a normal FP16 number down to 2^-25 of s, so the pair
// keeps about 22 significant bits across the FP32 range (a plain hi + lo pair
// would lose them below FP16's normal range).
//
// One persistent CTA per SM, 320 threads in five roles:
//   warp 0      producer: cp.async.bulk.tensor loads of the A planes of each
//               64-row K chunk into a ring of shared-memory slots (128-byte swizzle)
//   warp 1      allocates tensor memory; one lane issues tcgen05.mma and
//               tcgen05.commit (slot release, accumulator ready)
//   warps 2-3,
//   8-9         B operand: the chunk's 64 FP32 rows (bulk-copied by the
//               producer with the A planes), scaled, split, stored swizzled
//   warps 4-7   epilogue: tcgen05.ld of the two accumulators, combine, scale,
//               store (warp 4 + q reads tensor-memory lanes 32 q .. 32 q + 31)
// Every 64-row K chunk accumulates into a fresh pair of tensor-memory
// accumulators (double-buffered), which the epilogue adds into per-row FP32
// sums with round-to-nearest: the tensor cores truncate when they accumulate,
// and restarting every four MMA steps keeps that error at a few 2^-24 of each
// chunk's sum instead of growing with the panel's length. Every wait is bounded; on expiry the kernel records an error in
// the handle's error word, waits (bounded) for its own copies and MMAs, frees
// its tensor memory and returns.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "internal.cuh"
#include "tcgen05.cuh"

namespace hd {
namespace {

constexpr int kTcThreads = 320;
constexpr int kTcKC = 64;                   // K rows per ring slot
constexpr int kTcStages = 4;                // ring slots
constexpr int kPlaneBytes = kTcKC * 128;    // one 64-row plane of 128-byte rows
constexpr int kSlotA = 4 * kPlaneBytes;     // (piece, half) planes
constexpr int kSlotB32 = kTcKC * kTcR * 4;    // the chunk's FP32 B rows, bulk-copied, then converted in place
constexpr int kSlotBytes = kSlotA + kSlotB32;  // A planes + B (FP32 rows, then the FP16 high and low planes)
constexpr int kZeroBytes = kPlaneBytes;     // zero half for 64-row panels
constexpr int kTcSmem = kTcStages * kSlotBytes + kZeroBytes + 1024;
constexpr int kTmemCols = 256;              // two buffers x (D_hi, D_lo) x 64 columns

static_assert(kTcSmem <= 232448, "tensor-core apply exceeds the shared-memory limit");
static_assert(sizeof(TcPanel) == 56, "TcPanel layout");

// Arguments of one apply stage.
struct TcArgs {
  const TcPanel* panels;
  const int32_t* cta;       // panel ranges per CTA
  const float* B;           // FP32 rows of kTcR values: x_t (V) or t (U)
  const float* colmax;      // kTcR column maxima of |x_t| (bits of non-negative floats)
  const int32_t* vmap;      // V: column -> t index
  const float* fac;         // V: per t index su * sv
  const float* wbox;        // U: per scale box, power of two bounding |t| / sigma_x
  float* out;               // V: t (rows of kTcR); U: level slices of y (rows of kTcR)
  float* part;              // U: partial sums of cut panels (128-row blocks of kTcR)
  int64_t N;                // U: points (the slice stride)
};

template <bool VMODE>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_apply(const __grid_constant__ CUtensorMap tmap, TcArgs a,
                                                            int32_t* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tc_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* zero = sm + kTcStages * kSlotBytes;
  __shared__ __align__(8) uint64_t full_a[kTcStages], full_b[kTcStages], empty[kTcStages], dfull[2], dempty[2], fin;
  __shared__ uint32_t tmem_base;
  __shared__ float sx[kTcR];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int p0 = a.cta[blockIdx.x], p1 = a.cta[blockIdx.x + 1];

  for (int i = tid; i < kZeroBytes / 16; i += kTcThreads) reinterpret_cast<uint4*>(zero)[i] = make_uint4(0, 0, 0, 0);
  if (tid < kTcR) sx[tid] = pow2_above(a.colmax[tid]);
  if (tid == 0) {
    for (int i = 0; i < kTcStages; ++i) {
      bar_init(&full_a[i], 1);
      bar_init(&full_b[i], 4);  // one arrival per B warp
      bar_init(&empty[i], 1);   // tcgen05.commit
    }
    for (int i = 0; i < 2; ++i) {
      bar_init(&dfull[i], 1);
      bar_init(&dempty[i], 4);  // one arrival per epilogue warp
    }
    bar_init(&fin, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the zero half, read by the tensor cores
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  bool ok = true;

  if (warp == 0) {
    // producer: A planes of every K chunk
    if (lane == 0) {
      int64_t s = 0;
      for (int p = p0; p < p1 && ok; ++p) {
        const TcPanel P = a.panels[p];
        const int nk = (P.K + kTcKC - 1) / kTcKC;
        for (int kc = 0; kc < nk; ++kc, ++s) {
          const int slot = (int)(s % kTcStages);
          if (s >= kTcStages && !(ok = bar_wait(&empty[slot], (uint32_t)((s / kTcStages - 1) & 1), err, 0))) break;
          unsigned char* base = sm + slot * kSlotBytes;
          // the chunk's valid B rows (FP32, contiguous) ride on the same barrier
          const int nb = max(0, min(kTcKC, P.kvalid - kc * kTcKC));
          bar_expect(&full_a[slot], (uint32_t)(P.pieces * P.halves * kPlaneBytes + nb * kTcR * 4));
          if (nb > 0)
            bulk_load(base + kSlotA, a.B + ((int64_t)P.brow + (int64_t)kc * kTcKC) * kTcR,
                      (uint32_t)(nb * kTcR * 4), &full_a[slot]);
          for (int pc = 0; pc < P.pieces; ++pc)
            for (int hh = 0; hh < P.halves; ++hh) {
              const int64_t y = P.arow + (int64_t)(pc * P.halves + hh) * P.kstride + P.koff + (int64_t)kc * kTcKC;
              tma_load(base + (pc * 2 + hh) * kPlaneBytes, &tmap, 0, (int)y, &full_a[slot]);
            }
        }
      }
      // the loads issued last have landed before the CTA may exit (at once,
      // unless a wait above expired)
      for (int64_t t = s > kTcStages ? s - kTcStages : 0; t < s; ++t)
        bar_wait(&full_a[t % kTcStages], (uint32_t)((t / kTcStages) & 1), err, 7);
    }
  } else if (warp == 1) {
    // MMA issue: every K chunk into a fresh accumulator pair D(j & 1), j the
    // CTA's chunk count (the epilogue adds the chunk sums with round-to-nearest
    // FP32 additions, so the tensor cores' truncating accumulation spans four
    // MMA steps only)
    if (lane == 0) {
      const uint32_t zaddr = saddr(zero);
      int64_t s = 0;
      for (int p = p0; p < p1 && ok; ++p) {
        const TcPanel P = a.panels[p];
        const int nk = (P.K + kTcKC - 1) / kTcKC;
        for (int kc = 0; kc < nk; ++kc, ++s) {
          const int slot = (int)(s % kTcStages);
          const uint32_t ph = (uint32_t)((s / kTcStages) & 1);
          const int buf = (int)(s & 1);
          if (s >= 2 && !(ok = bar_wait(&dempty[buf], (uint32_t)((s / 2 - 1) & 1), err, 1))) break;
          if (!(ok = bar_wait(&full_a[slot], ph, err, 2) && bar_wait(&full_b[slot], ph, err, 3))) break;
          tc_fence_after();
          const uint32_t dhi = tmem + buf * 128, dlo = dhi + 64;
          const uint32_t base = saddr(sm + slot * kSlotBytes);
          // a 64-row panel reads its second M half from the zero page
          const uint32_t lbo_hi = P.halves == 2 ? (uint32_t)kPlaneBytes : zaddr - base;
          const uint32_t lbo_lo = P.halves == 2 ? (uint32_t)kPlaneBytes : zaddr - (base + 2 * kPlaneBytes);
          const int krem = P.K - kc * kTcKC;
          const int ksteps = (krem < kTcKC ? krem : kTcKC) / 16;
          for (int ks = 0; ks < ksteps; ++ks) {
            const uint32_t off = (uint32_t)ks * 2048u;  // 16 rows of 128 bytes
            const uint64_t ah = smem_desc(base + off, lbo_hi, 1024);
            const uint64_t bh = smem_desc(base + kSlotA + off, kPlaneBytes, 1024);
            const uint64_t bl = smem_desc(base + kSlotA + kPlaneBytes + off, kPlaneBytes, 1024);
            const uint32_t acc = ks != 0 ? 1u : 0u;
            mma_f16(dhi, ah, bh, acc);
            mma_f16(dlo, ah, bl, acc);
            if (P.pieces == 2) mma_f16(dlo, smem_desc(base + 2 * kPlaneBytes + off, lbo_lo, 1024), bh, 1u);
          }
          mma_commit(&empty[slot]);  // the slot is free once these MMAs have read it
          mma_commit(&dfull[buf]);   // the chunk's sums are ready
        }
      }
      // every MMA of this CTA has completed before its tensor memory is freed
      mma_commit(&fin);
      bar_wait(&fin, 0, err, 4);
    }
  } else if (warp < 4 || warp >= 8) {
    // B operand: rows of kTcR FP32 values, scaled per column, split into FP16
    // high and low planes in the 128-byte swizzled layout (16-byte chunk c of
    // row r at chunk c ^ (r & 7)); four warps, eight 4-column items per thread
    const int ct = warp < 4 ? tid - 64 : tid - 192;  // 0 .. 127
    const int q4 = ct & 15;                          // this thread's four columns 4 q4 .. 4 q4 + 3
    int64_t s = 0;
    for (int p = p0; p < p1 && ok; ++p) {
      const TcPanel P = a.panels[p];
      const float wb = VMODE ? 1.f : a.wbox[P.sbox];
      float2 inv01, inv23;  // powers of two: exact
      inv01.x = 1.f / (wb * sx[4 * q4]);
      inv01.y = 1.f / (wb * sx[4 * q4 + 1]);
      inv23.x = 1.f / (wb * sx[4 * q4 + 2]);
      inv23.y = 1.f / (wb * sx[4 * q4 + 3]);
      const int nk = (P.K + kTcKC - 1) / kTcKC;
      for (int kc = 0; kc < nk; ++kc, ++s) {
        const int slot = (int)(s % kTcStages);
        // the slot's loads have landed (the producer issued them after the
        // slot's previous MMAs had released it)
        if (!(ok = bar_wait(&full_a[slot], (uint32_t)((s / kTcStages) & 1), err, 5))) break;
        unsigned char* bh = sm + slot * kSlotBytes + kSlotA;
        unsigned char* bl = bh + kPlaneBytes;
        const float* b32 = reinterpret_cast<const float*>(bh);
        const int kv = P.kvalid - kc * kTcKC;  // rows with data in this chunk
        // all four warps read their FP32 items before any FP16 plane overwrites them
        float4 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int r = (ct >> 4) + 8 * j;
          v[j] = r < kv ? *reinterpret_cast<const float4*>(b32 + r * kTcR + 4 * q4) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int r = (ct >> 4) + 8 * j;
          const float2 a01 = make_float2(v[j].x * inv01.x, v[j].y * inv01.y);
          const float2 a23 = make_float2(v[j].z * inv23.x, v[j].w * inv23.y);
          const __half2 h01 = __float22half2_rn(a01), h23 = __float22half2_rn(a23);
          const float2 f01 = __half22float2(h01), f23 = __half22float2(h23);
          const __half2 l01 = __float22half2_rn(make_float2((a01.x - f01.x) * kLoScale, (a01.y - f01.y) * kLoScale));
          const __half2 l23 = __float22half2_rn(make_float2((a23.x - f23.x) * kLoScale, (a23.y - f23.y) * kLoScale));
          const int phys = r * 128 + ((((q4 >> 1) ^ (r & 7))) << 4) + (q4 & 1) * 8;
          *reinterpret_cast<uint2*>(bh + phys) =
              make_uint2(*reinterpret_cast<const uint32_t*>(&h01), *reinterpret_cast<const uint32_t*>(&h23));
          *reinterpret_cast<uint2*>(bl + phys) =
              make_uint2(*reinterpret_cast<const uint32_t*>(&l01), *reinterpret_cast<const uint32_t*>(&l23));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
        __syncwarp();
        if (lane == 0) bar_arrive(&full_b[slot]);
      }
    }
  } else {
    // epilogue: tensor-memory lanes 32 qw .. 32 qw + 31 = D rows of this warp;
    // each K chunk's D_hi + 2^-11 D_lo is added into the row's running sums
    const int qw = warp - 4;
    const int r = qw * 32 + lane;
    int64_t s = 0;
    for (int p = p0; p < p1 && ok; ++p) {
      const TcPanel P = a.panels[p];
      const int nk = (P.K + kTcKC - 1) / kTcKC;
      // the row's output address and scale, loaded before the chunks arrive
      float* dst = nullptr;
      float f = 0.f;
      if (r < P.mvalid) {
        if constexpr (VMODE) {
          const int32_t t = a.vmap[P.out0 + r];
          f = a.fac[t];
          dst = a.out + (int64_t)t * kTcR;
        } else {
          f = a.wbox[P.sbox];
          dst = P.part >= 0 ? a.part + ((int64_t)P.part * 128 + r) * kTcR
                            : a.out + ((int64_t)P.slice * a.N + P.out0 + r) * kTcR;
        }
      }
      float tot[kTcR];
#pragma unroll
      for (int i = 0; i < kTcR; ++i) tot[i] = 0.f;
      for (int kc = 0; kc < nk; ++kc, ++s) {
        const int buf = (int)(s & 1);
        if (!(ok = bar_wait(&dfull[buf], (uint32_t)((s / 2) & 1), err, 6))) break;
        tc_fence_after();
        const uint32_t dhi = tmem + buf * 128 + ((uint32_t)(qw * 32) << 16), dlo = dhi + 64;
#pragma unroll
        for (int c0 = 0; c0 < kTcR; c0 += 16) {
          float hv[16], lv[16];
          tmem_ld16(dhi + c0, hv);
          tmem_ld16(dlo + c0, lv);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) tot[c0 + j] += fmaf(lv[j], 1.f / kLoScale, hv[j]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) bar_arrive(&dempty[buf]);
      }
      if (!ok) break;
      if (r < P.mvalid) {
#pragma unroll
        for (int j = 0; j < kTcR; j += 4) {
          float4 o;
          o.x = f * sx[j] * tot[j];
          o.y = f * sx[j + 1] * tot[j + 1];
          o.z = f * sx[j + 2] * tot[j + 2];
          o.w = f * sx[j + 3] * tot[j + 3];
          *reinterpret_cast<float4*>(dst + j) = o;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

}  // namespace
}  // namespace hd

namespace hd {
namespace {

// ------------------------------------------------------------------ packing ----
// Per factor column t (one warp each): max |U|, max |V|, sum |V| and
// ||u|| ||v|| of the FP64 ACA factors.
__global__ void k_tc_colstats(int64_t ncol, const int64_t* __restrict__ colU, const int64_t* __restrict__ colV,
                              const int32_t* __restrict__ rows_u, const int32_t* __restrict__ rows_v,
                              const double* __restrict__ U64, const double* __restrict__ V64,
                              double4* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = warp; c < ncol; c += nw) {
    double mu = 0.0, mv = 0.0, sv = 0.0, nu = 0.0, nv = 0.0;
    for (int i = lane; i < rows_u[c]; i += 32) {
      const double v = U64[colU[c] + i];
      mu = fmax(mu, fabs(v));
      nu = fma(v, v, nu);
    }
    for (int i = lane; i < rows_v[c]; i += 32) {
      const double v = V64[colV[c] + i];
      mv = fmax(mv, fabs(v));
      sv += fabs(v);
      nv = fma(v, v, nv);
    }
    for (int o = 16; o; o >>= 1) {
      mu = fmax(mu, __shfl_xor_sync(0xffffffffu, mu, o));
      mv = fmax(mv, __shfl_xor_sync(0xffffffffu, mv, o));
      sv += __shfl_xor_sync(0xffffffffu, sv, o);
      nu += __shfl_xor_sync(0xffffffffu, nu, o);
      nv += __shfl_xor_sync(0xffffffffu, nv, o);
    }
    if (lane == 0) out[c] = make_double4(mu, mv, sv, sqrt(nu) * sqrt(nv));
  }
}

// The planes of every panel of one stream from the FP64 ACA output. V panels:
// row k = source point brow + k, entry j of half hh = V column out0 + 64 hh + j
// (its t index through vmap; zero outside the rows of the column's source box,
// since a panel may hold the columns of several consecutive small boxes). U panels: row k = t index brow + k, entry j of
// half hh = point out0 + 64 hh + j. Entries are divided by their column's
// power-of-two scale and split into the high and the scaled low FP16 part;
// rows >= kvalid and entries past mvalid are zero. One CTA per panel.
template <bool VMODE>
__global__ void __launch_bounds__(256) k_tc_pack(int64_t npan, const TcPanel* __restrict__ panels,
                                                 const int32_t* __restrict__ vmap, const int64_t* __restrict__ colU,
                                                 const int64_t* __restrict__ colV, const int32_t* __restrict__ urow0,
                                                 const int32_t* __restrict__ vrow0, const int32_t* __restrict__ vrows,
                                                 const double* __restrict__ U64, const double* __restrict__ V64,
                                                 const float* __restrict__ su, const float* __restrict__ sv,
                                                 __half* __restrict__ out) {
  for (int64_t p = blockIdx.x; p < npan; p += gridDim.x) {
    const TcPanel P = panels[p];
    const int64_t n = (int64_t)P.halves * P.kstride * 64;
    for (int64_t idx = threadIdx.x; idx < n; idx += blockDim.x) {
      const int hh = (int)(idx / ((int64_t)P.kstride * 64));
      const int k = (int)((idx / 64) % P.kstride), j = (int)(idx % 64);
      const int m = 64 * hh + j;
      double v = 0.0;
      if (k < P.kvalid && m < P.mvalid) {
        if constexpr (VMODE) {
          // packed panels hold several source boxes: a column is zero outside its own box's rows
          const int32_t t = vmap[P.out0 + m];
          const int64_t rr = (int64_t)P.brow + k - vrow0[t];
          if (rr >= 0 && rr < vrows[t]) v = V64[colV[t] + rr] / (double)sv[t];
        } else {
          const int32_t t = P.brow + k;
          v = U64[colU[t] + (P.out0 - urow0[t]) + m] / (double)su[t];
        }
      }
      const __half hi = __double2half(v);
      const __half lo = __double2half((v - (double)__half2float(hi)) * 2048.0);
      const int64_t row = P.arow + (int64_t)hh * P.kstride + k;
      out[row * 64 + j] = hi;
      if (P.pieces == 2) out[(row + (int64_t)P.halves * P.kstride) * 64 + j] = lo;
    }
  }
}

int64_t pad16(int64_t v) { return (v + 15) / 16 * 16; }

// Ranges of consecutive panels per CTA, balanced by the bytes they move (the
// factor planes, the B rows, the kTcR-wide output rows) plus a fixed cost per
// panel (the ring round trip and the epilogue): trees of many small boxes have
// many one-step panels whose output outweighs their planes.
void tc_schedule(TcStream& S, int ctas, double fixed = 32768.0) {
  std::vector<double> w(S.h_panels.size());
  double tot = 0.0;
  for (size_t i = 0; i < w.size(); ++i) {
    const TcPanel& P = S.h_panels[i];
    w[i] = (double)P.pieces * P.halves * P.K * 128.0 + (double)P.K * kTcR * 4.0 + (double)P.mvalid * kTcR * 4.0 +
           fixed;
    tot += w[i];
  }
  ctas = (int)std::max<int64_t>(1, std::min<int64_t>(ctas, (int64_t)w.size()));
  S.h_cta.assign(ctas + 1, (int32_t)w.size());
  S.h_cta[0] = 0;
  double acc = 0.0;
  int c = 1;
  for (size_t i = 0; i < w.size() && c < ctas; ++i) {
    acc += w[i];
    while (c < ctas && acc >= tot * c / ctas) S.h_cta[c++] = (int32_t)(i + 1);
  }
  S.ctas = ctas;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// A 2-D tensor map over the stream (64 FP16 per row, `rows` rows), boxes of
// 64 x kTcKC rows with the 128-byte swizzle the MMA descriptors expect; rows
// past the end read as zero.
int encode_tmap(TcStream& S) {
  static EncodeTiledFn fn = nullptr;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!fn) {
      void* p = nullptr;
      cudaDriverEntryPointQueryResult q;
      HD_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
      if (!p || q != cudaDriverEntryPointSuccess) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return HODLRDD_ERR_CUDA;
      }
      fn = reinterpret_cast<EncodeTiledFn>(p);
    }
  }
  static_assert(sizeof(CUtensorMap) == sizeof(S.tmap), "tensor map size");
  CUtensorMap tm;
  std::memset(&tm, 0, sizeof tm);
  const cuuint64_t gdim[2] = {64, (cuuint64_t)std::max<int64_t>(S.rows, 1)};
  const cuuint64_t gstr[1] = {128};
  const cuuint32_t box[2] = {64, (cuuint32_t)kTcKC};
  const cuuint32_t est[2] = {1, 1};
  const CUresult r = fn(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, S.data.p, gdim, gstr, box, est,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char buf[96];
    std::snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    set_error(buf);
    return HODLRDD_ERR_CUDA;
  }
  std::memcpy(S.tmap, &tm, sizeof tm);
  return HODLRDD_OK;
}

double pow2_above_host(double m) {
  if (!(m > 0.0)) return 1.0;
  int e = 0;
  std::frexp(m, &e);
  return std::ldexp(1.0, e);
}

}  // namespace

int64_t tc_device_bytes(const hodlrdd_s* h) {
  const Plan& P = h->plan;
  return (int64_t)(P.tcv.data.bytes() + P.tcu.data.bytes() + P.tcv.panels.bytes() + P.tcu.panels.bytes() +
                   P.tcv.cta.bytes() + P.tcu.cta.bytes() + P.tc_vmap.bytes() + P.tc_fac.bytes() +
                   P.tc_wbox.bytes() + P.tc_split.bytes() + P.tc_splitp.bytes());
}

// Builds both tensor-core streams from the FP64 ACA factors: column scales,
// V panels per (level, source box, 128 columns), U panels per (level, target
// box, 128 rows) cut along K where that balances the CTAs, and their planes.
int pack_tc(hodlrdd_s* h, const DevBuf<double>& U64, const DevBuf<double>& V64, const std::vector<int64_t>& uoff64,
            const std::vector<int64_t>& voff64) {
  cudaStream_t st = h->st;
  Plan& P = h->plan;
  const int64_t nblk = h->nblk, ncol = h->total_rank;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  if (ncol >= INT32_MAX || h->N * (int64_t)kTcR >= ((int64_t)1 << 40)) {
    set_error("problem too large for the tensor-core form's 32-bit indices");
    return HODLRDD_ERR_UNSUPPORTED;
  }
  // per t column: FP64 data offsets, rows, first output point of its U rows
  std::vector<int64_t> hcolU(std::max<int64_t>(ncol, 1)), hcolV(std::max<int64_t>(ncol, 1));
  std::vector<int32_t> hru(std::max<int64_t>(ncol, 1)), hrv(std::max<int64_t>(ncol, 1)), hur0(std::max<int64_t>(ncol, 1)),
      hvr0(std::max<int64_t>(ncol, 1));
  for (int64_t b = 0; b < nblk; ++b)
    for (int k = 0; k < h->h_rank[b]; ++k) {
      const int64_t t = h->h_toff[b] + k;
      hcolU[t] = uoff64[b] + (int64_t)k * h->h_bm[b];
      hcolV[t] = voff64[b] + (int64_t)k * h->h_bn[b];
      hru[t] = h->h_bm[b];
      hrv[t] = h->h_bn[b];
      hur0[t] = h->h_bI0[b];
      hvr0[t] = h->h_bJ0[b];
    }
  DevBuf<int64_t> colU, colV;
  DevBuf<int32_t> ru, rv, ur0, vr0;
  HD_TRY(upload(colU, hcolU, st));
  HD_TRY(upload(colV, hcolV, st));
  HD_TRY(upload(ru, hru, st));
  HD_TRY(upload(rv, hrv, st));
  HD_TRY(upload(ur0, hur0, st));
  HD_TRY(upload(vr0, hvr0, st));
  std::vector<double4> stats(std::max<int64_t>(ncol, 1), make_double4(0, 0, 0, 0));
  if (ncol > 0) {
    DevBuf<double4> dstats;
    HD_TRY(dstats.alloc(ncol));
    k_tc_colstats<<<std::max(1, std::min<int>((int)((ncol + 7) / 8), sms * 16)), 256, 0, st>>>(
        ncol, colU.p, colV.p, ru.p, rv.p, U64.p, V64.p, dstats.p);
    HD_CUDA(cudaGetLastError());
    HD_TRY(download(stats, dstats.p, (size_t)ncol, st));
    HD_CUDA(cudaStreamSynchronize(st));
  }
  std::vector<float> hsu(std::max<int64_t>(ncol, 1), 1.f), hsv(std::max<int64_t>(ncol, 1), 1.f),
      hfac(std::max<int64_t>(ncol, 1), 1.f);
  for (int64_t t = 0; t < ncol; ++t) {
    hsu[t] = (float)pow2_above_host(stats[t].x);
    hsv[t] = (float)pow2_above_host(stats[t].y);
    hfac[t] = hsu[t] * hsv[t];
  }
  // ---- V panels: per level and source box, the columns of its low-rank blocks
  TcStream& SV = P.tcv;
  SV = TcStream();
  std::vector<int32_t> hvmap;
  {
    std::vector<std::vector<int64_t>> by_src;
    for (int l = 1; l <= h->kappa; ++l) {
      const Level& L = h->lv[l];
      by_src.assign(L.nb, {});
      for (int64_t b = h->h_blk_off[l]; b < h->h_blk_off[l + 1]; ++b)
        if (!h->h_dense[b] && h->h_rank[b] > 0) by_src[h->h_bsj[b]].push_back(b);
      // consecutive small source boxes share a panel (block-diagonal planes:
      // each column is zero outside its box's rows) when that streams fewer
      // bytes than their own panels, counting each panel's fixed cost
      auto cost = [](int64_t rows, int64_t cols) {
        return pad16(rows) * ((cols + 63) / 64) * 256 + 8192;
      };
      std::vector<int64_t> grp;
      int64_t grows = 0, gcols = 0;
      auto box_cols = [&](int64_t J) {
        int64_t c = 0;
        for (int64_t b : by_src[J]) c += h->h_rank[b];
        return c;
      };
      auto emit = [&](const std::vector<int64_t>& boxes) {
        const int32_t c0 = (int32_t)hvmap.size();
        for (int64_t J : boxes)
          for (int64_t b : by_src[J])
            for (int k = 0; k < h->h_rank[b]; ++k) hvmap.push_back((int32_t)(h->h_toff[b] + k));
        const int32_t cols = (int32_t)hvmap.size() - c0;
        const int32_t r0 = L.h_bstart[boxes.front()];
        const int32_t n = L.h_bstart[boxes.back() + 1] - r0;
        for (int32_t m0 = 0; m0 < cols; m0 += 128) {
          TcPanel Q{};
          Q.mvalid = std::min(128, cols - m0);
          Q.halves = Q.mvalid > 64 ? 2 : 1;
          Q.pieces = 2;
          Q.kstride = (int32_t)pad16(n);
          Q.K = Q.kstride;
          Q.koff = 0;
          Q.kvalid = n;
          Q.brow = r0;
          Q.out0 = c0 + m0;
          Q.sbox = 0;
          Q.slice = l - 1;
          Q.part = -1;
          Q.arow = SV.rows;
          SV.rows += (int64_t)Q.pieces * Q.halves * Q.kstride;
          SV.h_panels.push_back(Q);
        }
      };
      auto flush = [&]() {
        if (!grp.empty()) emit(grp);
        grp.clear();
        grows = gcols = 0;
      };
      for (int64_t J = 0; J < L.nb; ++J) {
        if (by_src[J].empty()) {
          flush();  // the group's rows must stay contiguous
          continue;
        }
        const int64_t nJ = L.h_bstart[J + 1] - L.h_bstart[J], cJ = box_cols(J);
        if (nJ > 64 || cJ > 128) {
          flush();
          emit({J});
          continue;
        }
        if (!grp.empty() && grows + nJ <= 64 && gcols + cJ <= 128 &&
            cost(grows + nJ, gcols + cJ) <= cost(grows, gcols) + cost(nJ, cJ)) {
          grp.push_back(J);
          grows += nJ;
          gcols += cJ;
          continue;
        }
        flush();
        grp.push_back(J);
        grows = nJ;
        gcols = cJ;
      }
      flush();
    }
  }
  // ---- U panels: per level and target box, its rows in tiles of 128, K over its t columns
  TcStream& SU = P.tcu;
  SU = TcStream();
  std::vector<float> hwbox;
  std::vector<TcPanel> whole;
  for (int l = 1; l <= h->kappa; ++l) {
    const Level& L = h->lv[l];
    for (int64_t I = 0; I < L.nb; ++I) {
      const int64_t b0 = h->h_blk_off[l] + L.h_iloff[I], b1 = h->h_blk_off[l] + L.h_iloff[I + 1];
      if (b1 <= b0) continue;
      const int64_t t0 = h->h_toff[b0], t1 = h->h_toff[b1 - 1] + h->h_rank[b1 - 1];
      if (t1 <= t0) continue;
      double wmax = 0.0;  // bound of |t| / sigma_x over the box's columns: su ||V||_1
      for (int64_t t = t0; t < t1; ++t) wmax = std::max(wmax, (double)hsu[t] * stats[t].z);
      const int32_t sbox = (int32_t)hwbox.size();
      hwbox.push_back((float)pow2_above_host(wmax));
      const int32_t m = L.h_bstart[I + 1] - L.h_bstart[I];
      for (int32_t r0 = 0; r0 < m; r0 += 128) {
        TcPanel Q{};
        Q.mvalid = std::min(128, m - r0);
        Q.halves = Q.mvalid > 64 ? 2 : 1;
        Q.pieces = 2;
        Q.kstride = (int32_t)pad16(t1 - t0);
        Q.K = Q.kstride;
        Q.koff = 0;
        Q.kvalid = (int32_t)(t1 - t0);
        Q.brow = (int32_t)t0;
        Q.out0 = L.h_bstart[I] + r0;
        Q.sbox = sbox;
        Q.slice = l - 1;
        Q.part = -1;
        Q.arow = SU.rows;
        SU.rows += (int64_t)Q.pieces * Q.halves * Q.kstride;
        whole.push_back(Q);
      }
    }
  }
  if (SV.rows >= INT32_MAX - kTcKC || SU.rows >= INT32_MAX - kTcKC) {
    set_error("factor streams too large for 32-bit tensor-map coordinates");
    return HODLRDD_ERR_UNSUPPORTED;
  }
  // pack the planes (from the whole U panels, before any cut)
  HD_TRY(SV.data.alloc((size_t)std::max<int64_t>(SV.rows, 1) * 64));
  HD_TRY(SU.data.alloc((size_t)std::max<int64_t>(SU.rows, 1) * 64));
  DevBuf<int32_t> dvmap;
  DevBuf<float> dsu, dsv;
  HD_TRY(upload(P.tc_vmap, hvmap.empty() ? std::vector<int32_t>{0} : hvmap, st));
  HD_TRY(upload(dsu, hsu, st));
  HD_TRY(upload(dsv, hsv, st));
  HD_TRY(upload(P.tc_fac, hfac, st));
  HD_TRY(upload(P.tc_wbox, hwbox.empty() ? std::vector<float>{1.f} : hwbox, st));
  {
    DevBuf<TcPanel> tmpv, tmpu;
    HD_TRY(upload(tmpv, SV.h_panels, st));
    HD_TRY(upload(tmpu, whole, st));
    if (!SV.h_panels.empty())
      k_tc_pack<true><<<(int)std::min<size_t>(SV.h_panels.size(), 65535), 256, 0, st>>>(
          (int64_t)SV.h_panels.size(), tmpv.p, P.tc_vmap.p, colU.p, colV.p, ur0.p, vr0.p, rv.p, U64.p, V64.p,
          dsu.p, dsv.p, SV.data.p);
    if (!whole.empty())
      k_tc_pack<false><<<(int)std::min<size_t>(whole.size(), 65535), 256, 0, st>>>(
          (int64_t)whole.size(), tmpu.p, P.tc_vmap.p, colU.p, colV.p, ur0.p, vr0.p, rv.p, U64.p, V64.p,
          dsu.p, dsv.p, SU.data.p);
    HD_CUDA(cudaGetLastError());
    HD_CUDA(cudaStreamSynchronize(st));
  }
  // cut long U panels along K (multiples of the K chunk) so that CTAs get
  // balanced work; their partial sums are added in order by k_tc_combine
  {
    double tot = 0.0;
    for (const TcPanel& Q : whole) tot += (double)Q.pieces * Q.halves * Q.K;
    const double cap = std::max(tot / (4.0 * sms), 4.0 * kTcKC);
    P.h_tc_split.clear();
    P.h_tc_splitp.clear();
    P.tc_parts = 0;
    for (const TcPanel& Q : whole) {
      const double rowsq = (double)Q.pieces * Q.halves * Q.K;
      const int nsplit = (int)std::min<double>(std::ceil(rowsq / cap), (double)((Q.K + kTcKC - 1) / kTcKC));
      if (nsplit <= 1) {
        SU.h_panels.push_back(Q);
        continue;
      }
      const int32_t chunk = (int32_t)((Q.K / kTcKC + nsplit - 1) / nsplit) * kTcKC;
      const int32_t first = (int32_t)P.tc_parts;
      int n = 0;
      for (int32_t k0 = 0; k0 < Q.K; k0 += chunk, ++n) {
        TcPanel S2 = Q;
        S2.koff = k0;
        S2.K = std::min(chunk, Q.K - k0);
        S2.kvalid = std::max(0, std::min(Q.kvalid - k0, S2.K));
        S2.brow = Q.brow + k0;
        S2.part = first + n;
        SU.h_panels.push_back(S2);
      }
      P.tc_parts += n;
      P.h_tc_split.push_back(make_int2(first, n));
      P.h_tc_splitp.push_back((int32_t)(SU.h_panels.size() - n));  // its first sub-panel carries out0, mvalid, slice
    }
  }
  tc_schedule(SV, sms);
  tc_schedule(SU, sms);
  HD_TRY(upload(SV.panels, SV.h_panels.empty() ? std::vector<TcPanel>{TcPanel{}} : SV.h_panels, st));
  HD_TRY(upload(SU.panels, SU.h_panels.empty() ? std::vector<TcPanel>{TcPanel{}} : SU.h_panels, st));
  HD_TRY(upload(SV.cta, SV.h_cta, st));
  HD_TRY(upload(SU.cta, SU.h_cta, st));
  HD_TRY(upload(P.tc_split, P.h_tc_split.empty() ? std::vector<int2>{make_int2(0, 0)} : P.h_tc_split, st));
  HD_TRY(upload(P.tc_splitp, P.h_tc_splitp.empty() ? std::vector<int32_t>{0} : P.h_tc_splitp, st));
  HD_TRY(encode_tmap(SV));
  HD_TRY(encode_tmap(SU));
  h->factor_bytes = (SV.rows + SU.rows) * 128;
  P.tc_tail_cols = 0;
  HD_CUDA(cudaStreamSynchronize(st));
  return HODLRDD_OK;
}

namespace {

// x_t[i][c] = x[perm[i]][c0 + c] for c < nr, 0 for nr <= c < kTcR; and the
// column maxima of |x_t| (non-negative floats compare as their bits).
__global__ void k_tc_gather(const float* __restrict__ x, const int32_t* __restrict__ perm, int64_t N, int ldx, int c0,
                            int nr, float* __restrict__ xt, unsigned int* __restrict__ colmax) {
  __shared__ unsigned int smax[kTcR];
  if (threadIdx.x < kTcR) smax[threadIdx.x] = 0u;
  __syncthreads();
  const int c = threadIdx.x % kTcR;
  unsigned int m = 0u;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N * kTcR; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / kTcR;
    const float v = c < nr ? x[(int64_t)perm[i] * ldx + c0 + c] : 0.f;
    xt[e] = v;
    m = max(m, __float_as_uint(fabsf(v)));
  }
  atomicMax(&smax[c], m);
  __syncthreads();
  if (threadIdx.x < kTcR) atomicMax(&colmax[threadIdx.x], smax[threadIdx.x]);
}

// Sums of cut U panels: y_l rows of the panel = sum of its sub-panels' partials, in order.
__global__ void k_tc_combine(int64_t nsplit, const int2* __restrict__ split, const int32_t* __restrict__ splitp,
                             const TcPanel* __restrict__ panels, const float* __restrict__ part, int64_t N,
                             float* __restrict__ ylev) {
  for (int64_t s = blockIdx.x; s < nsplit; s += gridDim.x) {
    const int2 sp = split[s];
    const TcPanel P = panels[splitp[s]];
    for (int e = threadIdx.x; e < P.mvalid * kTcR; e += blockDim.x) {
      const int r = e / kTcR, c = e % kTcR;
      float acc = 0.f;
      for (int i = 0; i < sp.y; ++i) acc += part[((int64_t)(sp.x + i) * 128 + r) * kTcR + c];
      ylev[((int64_t)P.slice * N + P.out0 + r) * kTcR + c] = acc;
    }
  }
}

// y[perm[i]][c0 + c] = near(i, c) + sum over the level slices of y_l(i, c), c < nr.
__global__ void k_tc_finish(const float* __restrict__ ynear, const float* __restrict__ ylev, int slices, int64_t N,
                            const int32_t* __restrict__ perm, float* __restrict__ y, int ldy, int c0, int nr) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N * kTcR; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % kTcR);
    if (c >= nr) continue;
    const int64_t i = e / kTcR;
    float acc = ynear[e];
    for (int l = 0; l < slices; ++l) acc += ylev[(int64_t)l * N * kTcR + e];
    y[(int64_t)perm[i] * ldy + c0 + c] = acc;
  }
}

int set_tc_attr() {
  static PerDeviceOnce once;
  return once.run([] {
    HD_CUDA(cudaFuncSetAttribute(k_tc_apply<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
    HD_CUDA(cudaFuncSetAttribute(k_tc_apply<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
    return (int)HODLRDD_OK;
  });
}

int tc_stage(bool vmode, const TcStream& S, const TcArgs& a, int32_t* err, cudaStream_t st) {
  if (S.h_panels.empty()) return HODLRDD_OK;
  CUtensorMap tm;
  std::memcpy(&tm, S.tmap, sizeof tm);
  if (vmode) k_tc_apply<true><<<S.ctas, kTcThreads, kTcSmem, st>>>(tm, a, err);
  else k_tc_apply<false><<<S.ctas, kTcThreads, kTcSmem, st>>>(tm, a, err);
  HD_CUDA(cudaGetLastError());
  return HODLRDD_OK;
}

}  // namespace

// y = K x for FP16X2 handles: chunks of kTcR right-hand sides; the near field
// runs as 16-wide FP32 tiles on the aux stream beside the tensor-core applies.
int launch_matvec_tc(hodlrdd_s* h, const float* x, float* y, int nrhs, cudaStream_t st) {
  HD_TRY(set_tc_attr());
  const Plan& P = h->plan;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  float* xt = reinterpret_cast<float*>(h->xt.p);
  float* t = reinterpret_cast<float*>(h->tbuf.p);
  float* yl = reinterpret_cast<float*>(h->ylev.p);
  float* pb = reinterpret_cast<float*>(h->pbuf.p);
  unsigned int* colmax = reinterpret_cast<unsigned int*>(pb + (size_t)std::max<int64_t>(P.tc_parts, 1) * 128 * kTcR);
  const int slices = std::max(h->kappa, 1);
  const int grid = (int)std::min<int64_t>((h->N * kTcR + 255) / 256, (int64_t)sms * 16);
  const bool prof = h->profiling;
  for (int c0 = 0; c0 < nrhs; c0 += kTcR) {
    const int nr = std::min(kTcR, nrhs - c0);
    cudaEvent_t ev[7];
    if (prof) {
      // the same five + two events per chunk as the other precisions
      for (int i = 0; i < 7; ++i) {
        if (h->ev_pool.empty()) {
          cudaEvent_t e;
          HD_CUDA(cudaEventCreate(&e));
          h->ev_pool.push_back(e);
        }
        ev[i] = h->ev_pool.back();
        h->ev_pool.pop_back();
      }
      h->ev_pending.emplace_back(ev, ev + 7);
      HD_CUDA(cudaEventRecord(ev[0], st));
    }
    HD_CUDA(cudaMemsetAsync(colmax, 0, kTcR * sizeof(unsigned int), st));
    k_tc_gather<<<grid, 256, 0, st>>>(x, h->perm.p, h->N, nrhs, c0, nr, xt, colmax);
    h->launches += 1;
    if (prof) HD_CUDA(cudaEventRecord(ev[1], st));
    // the near field needs x_t only: it runs on the aux stream beside the
    // applies; it is enqueued after the V-apply, so that the persistent
    // apply CTAs are placed first and the near-field CTAs fill the room left
    HD_CUDA(cudaEventRecord(h->ev_fork, st));
    HD_CUDA(cudaMemsetAsync(yl, 0, (size_t)slices * h->N * kTcR * sizeof(float), st));
    TcArgs av{P.tcv.panels.p, P.tcv.cta.p, xt, reinterpret_cast<const float*>(colmax), P.tc_vmap.p, P.tc_fac.p,
              P.tc_wbox.p, t, nullptr, h->N};
    HD_TRY(tc_stage(true, P.tcv, av, h->err.p, st));
    h->launches += P.tcv.h_panels.empty() ? 0 : 1;
    HD_CUDA(cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
    if (prof) HD_CUDA(cudaEventRecord(ev[5], h->aux));
    HD_CUDA(cudaMemsetAsync(h->ynear.p, 0, (size_t)h->N * kTcR * sizeof(float), h->aux));
    if (tc_near_supported(h)) {
      HD_TRY(launch_tc_near(h, h->aux, xt, colmax));
    } else {
      for (int cx = 0; cx < kTcR; cx += 16)
        if (cx < nr) HD_TRY(launch_tiles_nr(h, h->aux, xt, 16, kTcR, cx));
    }
    if (prof) HD_CUDA(cudaEventRecord(ev[6], h->aux));
    HD_CUDA(cudaEventRecord(h->ev_join, h->aux));
    if (prof) HD_CUDA(cudaEventRecord(ev[2], st));
    TcArgs au{P.tcu.panels.p, P.tcu.cta.p, t, reinterpret_cast<const float*>(colmax), P.tc_vmap.p, P.tc_fac.p,
              P.tc_wbox.p, yl, pb, h->N};
    HD_TRY(tc_stage(false, P.tcu, au, h->err.p, st));
    h->launches += P.tcu.h_panels.empty() ? 0 : 1;
    if (!P.h_tc_split.empty()) {
      k_tc_combine<<<(int)std::min<size_t>(P.h_tc_split.size(), 65535), 256, 0, st>>>(
          (int64_t)P.h_tc_split.size(), P.tc_split.p, P.tc_splitp.p, P.tcu.panels.p, pb, h->N, yl);
      h->launches += 1;
    }
    if (prof) HD_CUDA(cudaEventRecord(ev[3], st));
    HD_CUDA(cudaStreamWaitEvent(st, h->ev_join, 0));
    k_tc_finish<<<grid, 256, 0, st>>>(h->ynear.p, yl, h->kappa, h->N, h->perm.p, y, nrhs, c0, nr);
    h->launches += 1;
    if (prof) HD_CUDA(cudaEventRecord(ev[4], st));
    HD_CUDA(cudaGetLastError());
  }
  return HODLRDD_OK;
}

}  // namespace hd

namespace hd {

// One apply stage over an explicit panel set (a handle's, or a forest's).
int launch_tc_stage(bool vmode, const TcLaunch& L, int32_t* err, cudaStream_t st) {
  HD_TRY(set_tc_attr());
  const TcStream& S = *L.S;
  TcArgs a{S.panels.p, S.cta.p, L.B, reinterpret_cast<const float*>(L.colmax), L.vmap, L.fac, L.wbox, L.out, L.part,
           L.N};
  return tc_stage(vmode, S, a, err, st);
}

int launch_tc_combine(int64_t nsplit, const int2* split, const int32_t* splitp, const TcPanel* panels,
                      const float* part, int64_t N, float* ylev, cudaStream_t st) {
  if (nsplit <= 0) return HODLRDD_OK;
  k_tc_combine<<<(int)std::min<int64_t>(nsplit, 65535), 256, 0, st>>>(nsplit, split, splitp, panels, part, N, ylev);
  HD_CUDA(cudaGetLastError());
  return HODLRDD_OK;
}

void tc_schedule_stream(TcStream& S, int ctas, double fixed) { tc_schedule(S, ctas, fixed); }

int tc_encode_tmap(TcStream& S) { return encode_tmap(S); }

}  // namespace hd
