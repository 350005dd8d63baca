// Factor packing (a6) and the HODLRdD matrix-vector product (a7 - a10).
//
// Algorithm 2 in GPU form, for a chunk of NR right-hand sides:
//   a7  gather    x_t[i] = x[perm[i]]                          (tree order)
//   a8  V-apply   t_b[k] = V_b[:,k] . x_t(J_b)  for every low-rank IL block
//       U-apply   y_l(i) = U_box(i)[r,:] . t_box  for every level l and box
//   a9  dense     K(I,J) x_t(J) evaluated on the fly: IL blocks flagged dense at
//                 coarse levels, then per leaf box the near field (self and d' >= 1
//                 neighbours) and the leaf-level dense IL blocks
//   a10 combine   y[perm[i]] = sum_l y_l(i) + near(i)
//
// Both low-rank applies are the same operation: dot products of contiguous
// factor segments with a vector. V is stored column by column; U is stored per
// (level, box) row-major over the concatenated columns of the box's IL blocks,
// so a box's rows read one contiguous t vector. Each factor array is a stream
// of 16-byte aligned segments, consumed by one persistent CTA per SM: a
// producer lane moves 32 KB stages with cp.async.bulk into a shared-memory ring
// guarded by mbarriers; consumer warps split every stage into lane teams sized
// to the segment length and reduce with shuffles. Every output has one writer
// and a fixed summation order (bitwise reproducible, no atomics on results).
// All waits are bounded; on timeout the kernel records an error and returns.
//
// 16-bit factors carry one power-of-two FP32 scale per column (exact
// rescaling); the V-apply folds the U and V scales of column k into t_b[k].
#include <algorithm>
#include <climits>
#include <cmath>

#include "internal.cuh"

namespace hd {

size_t elem_size(int precision) {
  switch (precision) {
    case HODLRDD_PREC_FP64: return 8;
    case HODLRDD_PREC_FP32: return 4;
    default: return 2;
  }
}

namespace {

constexpr int kStageBytes = 32768;
constexpr int kStages = 4;
constexpr int kConsumerWarps = 16;
constexpr int kSegThreads = 32 * (1 + kConsumerWarps);
constexpr int kPanelRows = 512;                // rows per U panel
constexpr int kGuard = 16;                        // zero elements around xt and t (per rhs)
constexpr long long kWaitCycles = 4000000000LL;  // about two seconds at GB300 clocks

enum { ERR_WAIT_FULL = 1, ERR_WAIT_EMPTY = 2, ERR_WAIT_DRAIN = 3 };

// ---------------------------------------------------------- element types ----
template <class T> struct Fac;
template <> struct Fac<double> {
  using acc = double;
  static constexpr int E = 2;  // elements per 16-byte chunk
  static constexpr bool scaled = false;
  __device__ static double from(double v) { return v; }
  __host__ static double to_host(double v) { return v; }
  __device__ static void chunk(const void* p, double (&v)[2]) {
    double2 q = *reinterpret_cast<const double2*>(p);
    v[0] = q.x; v[1] = q.y;
  }
};
template <> struct Fac<float> {
  using acc = float;
  static constexpr int E = 4;
  static constexpr bool scaled = false;
  __device__ static float from(double v) { return (float)v; }
  __host__ static double to_host(float v) { return v; }
  __device__ static void chunk(const void* p, float (&v)[4]) {
    float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
};
template <> struct Fac<__half> {
  using acc = float;
  static constexpr int E = 8;
  static constexpr bool scaled = true;
  __device__ static __half from(double v) { return __float2half_rn((float)v); }
  __host__ static double to_host(__half v) { return (double)__half2float(v); }
  __device__ static void chunk(const void* p, float (&v)[8]) {
    uint4 q = *reinterpret_cast<const uint4*>(p);
    const __half2* hh = reinterpret_cast<const __half2*>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float2 f = __half22float2(hh[i]);
      v[2 * i] = f.x; v[2 * i + 1] = f.y;
    }
  }
};
template <> struct Fac<__nv_bfloat16> {
  using acc = float;
  static constexpr int E = 8;
  static constexpr bool scaled = true;
  __device__ static __nv_bfloat16 from(double v) { return __float2bfloat16_rn((float)v); }
  __host__ static double to_host(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
  __device__ static void chunk(const void* p, float (&v)[8]) {
    uint4 q = *reinterpret_cast<const uint4*>(p);
    const __nv_bfloat162* hh = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float2 f = __bfloat1622float2(hh[i]);
      v[2 * i] = f.x; v[2 * i + 1] = f.y;
    }
  }
};

// E * NR consecutive vector values (16-byte aligned) into registers.
template <class Acc, int E, int NR>
__device__ __forceinline__ void load_vec(const Acc* __restrict__ p, Acc (&v)[E * NR]) {
  constexpr int PER = 16 / sizeof(Acc);
#pragma unroll
  for (int i = 0; i < E * NR; i += PER) {
    if constexpr (sizeof(Acc) == 4) {
      float4 q = *reinterpret_cast<const float4*>(p + i);
      v[i] = q.x; v[i + 1] = q.y; v[i + 2] = q.z; v[i + 3] = q.w;
    } else {
      double2 q = *reinterpret_cast<const double2*>(p + i);
      v[i] = q.x; v[i + 1] = q.y;
    }
  }
}

// ------------------------------------------------------------- mbarriers ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with the given parity; false (and the error word set) if
// it has not completed within kWaitCycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int32_t* err, int code) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) {
      atomicCAS(err, 0, code);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void consumer_bar() {
  asm volatile("bar.sync 1, %0;" ::"n"(32 * kConsumerWarps) : "memory");
}

// ------------------------------------------------------ segmented dot ----
// Stage kinds (decided on the host): "short" stages hold whole segments of at
// most kLongChunks 16-byte chunks from up to kGmax groups and are processed by
// lane teams of Stage::ts lanes over a flat list of the stage's segments;
// "long" stages (ts = 0) hold whole longer segments of one group, each shared
// by all consumer warps; "piece" stages hold part of a segment longer than a
// stage. The vector slice of every group that fits kVecBytes is bulk-copied
// next to the factor data (one right-hand side).
constexpr int kLongChunks = 512;  // longer segments: all consumer warps share each one
constexpr int kBatchChunks = 64;  // shorter segments: batched transpose-reduction (one right-hand side)
constexpr int kVecBytes = 20480;
constexpr int kGmax = 32;
struct SlotMeta {
  Stage st;
  SegGroup g[kGmax];
  int32_t voff[kGmax];      // byte offset of group i's vector slice in the slot, -1 if not staged
  int32_t sbeg[kGmax + 1];  // first stage-local segment of group i
  int32_t gpos[kGmax];      // element offset of group i's first segment in the stage
  int32_t s0[kGmax];        // index within group i of its first segment in the stage
  int32_t ubeg[kGmax + 1];  // batched V-apply: first work unit (W columns) of group i
};
constexpr int kMetaBytes = (int)((sizeof(SlotMeta) + 127) / 128 * 128);
constexpr int kSlotBytes = kStageBytes + kVecBytes + kMetaBytes;

template <class T, int NR>
__device__ __forceinline__ void write_out(int64_t o, const typename Fac<T>::acc (&acc)[NR],
                                          typename Fac<T>::acc* __restrict__ out, const float* __restrict__ sa,
                                          const float* __restrict__ sb) {
  using Acc = typename Fac<T>::acc;
  const Acc sc = sa ? (Acc)(sa[o] * sb[o]) : Acc(1);
#pragma unroll
  for (int r = 0; r < NR; ++r) out[o * NR + r] = acc[r] * sc;
}

template <class T, int NR>
__device__ __forceinline__ void dot_chunk(const char* fp, const typename Fac<T>::acc* vp,
                                          typename Fac<T>::acc (&acc)[NR]) {
  using Acc = typename Fac<T>::acc;
  constexpr int E = Fac<T>::E;
  Acc f[E];
  Fac<T>::chunk(fp, f);
  Acc v[E * NR];
  load_vec<Acc, E, NR>(vp, v);
#pragma unroll
  for (int e = 0; e < E; ++e)
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] += f[e] * v[e * NR + r];
}

// Short stage: teams of TS lanes take the stage's segments round-robin across
// group boundaries, SU segments in flight per team; a lane covers chunks
// tl, tl + TS, ... of its segment. Shuffle reduction within the team.
template <class T, int NR>
__device__ __forceinline__ void consume_short(const SlotMeta* meta, const char* base,
                                              const typename Fac<T>::acc* __restrict__ vec,
                                              typename Fac<T>::acc* __restrict__ out, const float* __restrict__ sa,
                                              const float* __restrict__ sb, int cw, int lane) {
  using Acc = typename Fac<T>::acc;
  constexpr int E = Fac<T>::E;
  constexpr int SU = NR == 1 ? 4 : 2;
  const int TS = meta->st.pad;
  const int S = meta->st.nseg;
  const int per_warp = 32 / TS;
  const int nteams = kConsumerWarps * per_warp;
  const int team = cw * per_warp + lane / TS;
  const int tl = lane % TS;
  int gi = 0;
  for (int b0 = 0; b0 < S; b0 += nteams * SU) {
    Acc acc[SU][NR];
    int64_t oidx[SU];
#pragma unroll
    for (int u = 0; u < SU; ++u) {
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[u][r] = Acc(0);
      oidx[u] = -1;
      const int q = b0 + u * nteams + team;
      if (q < S) {
        while (q >= meta->sbeg[gi + 1]) ++gi;
        const SegGroup& G = meta->g[gi];
        const int j = q - meta->sbeg[gi];
        const int C = G.L / E;
        const char* sp = base + ((int64_t)meta->gpos[gi] + (int64_t)j * G.L) * sizeof(T);
        const int vo = meta->voff[gi];
        const Acc* vsrc = vo >= 0 ? reinterpret_cast<const Acc*>(base + kStageBytes + vo) : vec + (int64_t)G.vec * NR;
#pragma unroll 4
        for (int c = tl; c < C; c += TS) dot_chunk<T, NR>(sp + (size_t)c * 16, vsrc + (int64_t)c * E * NR, acc[u]);
        oidx[u] = (int64_t)G.out0 + meta->s0[gi] + j;
      }
    }
    for (int o = TS >> 1; o > 0; o >>= 1)
#pragma unroll
      for (int u = 0; u < SU; ++u)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[u][r] += __shfl_xor_sync(0xffffffffu, acc[u][r], o);
    if (tl == 0) {
#pragma unroll
      for (int u = 0; u < SU; ++u)
        if (oidx[u] >= 0) write_out<T, NR>(oidx[u], acc[u], out, sa, sb);
    }
  }
}

// Long stage: all consumer warps share one segment at a time; warp sums meet in
// double-buffered shared memory (one consumer barrier per segment).
template <class T, int NR>
__device__ __forceinline__ void consume_long(const SlotMeta* meta, const char* base,
                                             const typename Fac<T>::acc* __restrict__ vec,
                                             typename Fac<T>::acc* __restrict__ out, const float* __restrict__ sa,
                                             const float* __restrict__ sb, int cw, int lane,
                                             typename Fac<T>::acc* part, int& pbuf) {
  using Acc = typename Fac<T>::acc;
  constexpr int E = Fac<T>::E;
  const SegGroup& G = meta->g[0];
  const int C = G.L / E;
  const int vo = meta->voff[0];
  const Acc* vsrc = vo >= 0 ? reinterpret_cast<const Acc*>(base + kStageBytes + vo) : vec + (int64_t)G.vec * NR;
  const int ct = cw * 32 + lane;
  for (int j = 0; j < meta->st.nseg; ++j) {
    const char* sp = base + (int64_t)j * G.L * sizeof(T);
    Acc acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = Acc(0);
#pragma unroll 4
    for (int c = ct; c < C; c += kConsumerWarps * 32) dot_chunk<T, NR>(sp + (size_t)c * 16, vsrc + (int64_t)c * E * NR, acc);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      Acc a = acc[r];
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) part[(pbuf * kConsumerWarps + cw) * NR + r] = a;
    }
    consumer_bar();
    if (cw == 0 && lane == 0) {
      Acc tot[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        tot[r] = Acc(0);
        for (int w = 0; w < kConsumerWarps; ++w) tot[r] += part[(pbuf * kConsumerWarps + w) * NR + r];
      }
      write_out<T, NR>((int64_t)G.out0 + meta->st.s + j, tot, out, sa, sb);
    }
    pbuf ^= 1;
  }
}

// Producer warp of the segment streams: per stage it waits for the slot to
// drain, writes the stage's metadata (group descriptors, per-group segment,
// element and work-unit prefixes, vector slice offsets) into the slot and
// issues the bulk copies of the factor data and of the staged vector slices,
// all completing on the slot's `full` barrier.
template <class T, int NR>
__device__ void produce_segment_stages(const T* __restrict__ F, const SegGroup* __restrict__ groups,
                                       const Stage* __restrict__ stages, int q0, int q1,
                                       const typename Fac<T>::acc* __restrict__ vec, char* smem, uint64_t* full,
                                       uint64_t* empty, int32_t* err, int lane) {
  using Acc = typename Fac<T>::acc;
  constexpr bool STAGE_VEC = NR == 1;
  int issued = 0;
  bool ok = true;
  for (int q = q0; q < q1; ++q, ++issued) {
    const int slot = issued % kStages;
    const int use = issued / kStages;
    if (use > 0) {
      int w = 1;
      if (lane == 0) w = mbar_wait(&empty[slot], (use - 1) & 1, err, ERR_WAIT_EMPTY) ? 1 : 0;
      if (!__shfl_sync(0xffffffffu, w, 0)) {
        ok = false;
        break;
      }
    }
    char* base = smem + (size_t)slot * kSlotBytes;
    SlotMeta* meta = reinterpret_cast<SlotMeta*>(base + kStageBytes + kVecBytes);
    const Stage st = stages[q];
    const bool in = lane < st.ng;
    SegGroup G{};
    if (in) G = groups[st.g + lane];
    // segments of group `lane` in this stage
    const int avail = in ? G.cnt - (lane == 0 ? st.s : 0) : 0;
    int sc_avail = avail;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, sc_avail, o);
      if (lane >= o) sc_avail += t;
    }
    const int before = sc_avail - avail;
    const int take = in ? max(0, min(avail, st.nseg - before)) : 0;
    const int W = st.pad > 0 ? st.pad : 1;
    const int units = (take + W - 1) / W;
    int sc_take = take, sc_pos = take * G.L, sc_units = units;
    const int vb =
        (in && STAGE_VEC && st.piece < 0 && G.L * (int)sizeof(Acc) <= kVecBytes) ? G.L * (int)sizeof(Acc) : 0;
    int sc_vb = vb;
    for (int o = 1; o < 32; o <<= 1) {
      const int a = __shfl_up_sync(0xffffffffu, sc_take, o);
      const int b = __shfl_up_sync(0xffffffffu, sc_pos, o);
      const int c = __shfl_up_sync(0xffffffffu, sc_vb, o);
      const int d = __shfl_up_sync(0xffffffffu, sc_units, o);
      if (lane >= o) {
        sc_take += a;
        sc_pos += b;
        sc_vb += c;
        sc_units += d;
      }
    }
    const int vtotal = __shfl_sync(0xffffffffu, sc_vb, 31);
    const int voff = sc_vb - vb;
    if (in) {
      meta->g[lane] = G;
      meta->voff[lane] = vb > 0 ? voff : -1;
      meta->sbeg[lane] = sc_take - take;
      meta->gpos[lane] = sc_pos - take * G.L;
      meta->s0[lane] = lane == 0 ? st.s : 0;
      meta->ubeg[lane] = sc_units - units;
      if (lane == st.ng - 1) {
        meta->sbeg[lane + 1] = sc_take;
        meta->ubeg[lane + 1] = sc_units;
      }
    }
    if (lane == 0) meta->st = st;
    __threadfence_block();
    __syncwarp();
    const uint32_t fbytes = (uint32_t)st.nelem * sizeof(T);
    if (lane == 0) mbar_expect_tx(&full[slot], fbytes + (uint32_t)vtotal);
    __syncwarp();
    if (lane == 0) bulk_g2s(base, F + st.off, fbytes, &full[slot]);
    if (vb > 0) bulk_g2s(base + kStageBytes + voff, vec + G.vec, (uint32_t)vb, &full[slot]);
  }
  if (!ok && lane == 0) {
    // drain: copies already issued must land before the CTA's smem goes away
    for (int k = max(0, issued - kStages); k < issued; ++k)
      mbar_wait(&full[k % kStages], (k / kStages) & 1, err, ERR_WAIT_DRAIN);
  }
}

// Sum W per-lane partial values across a team of W lanes (W a power of two,
// teams aligned within the warp); lane i of the team ends with the total of
// value i. Butterfly halving: W - 1 shuffles for W sums.
template <class Acc, int W>
__device__ __forceinline__ Acc transpose_reduce(Acc (&v)[32], int tl) {
#pragma unroll
  for (int off = W / 2; off >= 1; off >>= 1) {
    const bool upper = (tl & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      const Acc send = upper ? v[i] : v[i + off];
      const Acc keep = upper ? v[i + off] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return v[0];
}

// Batched V-apply of a short stage (one right-hand side): a work unit is W
// consecutive columns of one block. The W lanes of a team own fixed row chunks
// tl, tl + W, ... (up to KMAX), keep the matching x chunks in registers, and
// accumulate all W columns before one transpose reduction, so each column costs
// one shared-memory load per chunk and (W - 1) / W shuffles.
template <class T, int W, int KMAX>
__device__ __forceinline__ void consume_vbatch(const SlotMeta* meta, const char* base,
                                               typename Fac<T>::acc* __restrict__ out, const float* __restrict__ sa,
                                               const float* __restrict__ sb, int cw, int lane) {
  using Acc = typename Fac<T>::acc;
  constexpr int E = Fac<T>::E;
  constexpr int PER_WARP = 32 / W;
  constexpr int NTEAMS = kConsumerWarps * PER_WARP;
  const int tl = lane % W;
  const int ng = meta->st.ng;
  const int nunits = meta->ubeg[ng];
  int gi = 0;
  for (int u0 = cw * PER_WARP; u0 < nunits; u0 += NTEAMS) {
    const int u = u0 + lane / W;
    const bool valid = u < nunits;
    Acc acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = Acc(0);
    int ncols = 0;
    int64_t o0 = 0;
    if (valid) {
      while (u >= meta->ubeg[gi + 1]) ++gi;
      const SegGroup& G = meta->g[gi];
      const int C = G.L / E;
      const int j0 = (u - meta->ubeg[gi]) * W;
      const int take = meta->sbeg[gi + 1] - meta->sbeg[gi];
      ncols = min(W, take - j0);
      o0 = (int64_t)G.out0 + meta->s0[gi] + j0;
      const Acc* xs = reinterpret_cast<const Acc*>(base + kStageBytes + meta->voff[gi]);
      Acc xr[KMAX][E];
#pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        const int c = tl + k * W;
        if (c < C) {
          load_vec<Acc, E, 1>(xs + (int64_t)c * E, xr[k]);
        } else {
#pragma unroll
          for (int e = 0; e < E; ++e) xr[k][e] = Acc(0);
        }
      }
      const char* cp = base + ((int64_t)meta->gpos[gi] + (int64_t)j0 * G.L) * sizeof(T);
#pragma unroll
      for (int jj = 0; jj < W; ++jj) {
        if (jj < ncols) {
#pragma unroll
          for (int k = 0; k < KMAX; ++k) {
            const int c = tl + k * W;
            if (c < C) {
              Acc f[E];
              Fac<T>::chunk(cp + ((int64_t)jj * G.L + (int64_t)c * E) * sizeof(T), f);
#pragma unroll
              for (int e = 0; e < E; ++e) acc[jj] += f[e] * xr[k][e];
            }
          }
        }
      }
    }
    const Acc tot = transpose_reduce<Acc, W>(acc, tl);
    if (valid && tl < ncols) {
      const int64_t o = o0 + tl;
      const Acc sc = sa ? (Acc)(sa[o] * sb[o]) : Acc(1);
      out[o] = tot * sc;
    }
  }
}

// out[out0 + s] = scale(out0 + s) * sum_e F[seg s][e] vec[vec + e]  (x NR columns)
//
// Warp 0 produces: per stage it waits for the slot to drain, writes the stage's
// metadata (group descriptors, per-group segment and element prefixes, vector
// slice offsets) into the slot, and issues the bulk copies of the factor data
// and of the staged vector slices, all completing on the slot's `full`
// barrier. Consumer warps read only shared memory on their critical path.
template <class T, int NR>
__global__ void __launch_bounds__(kSegThreads, 1)
    k_segdot(const T* __restrict__ F, const SegGroup* __restrict__ groups, const Stage* __restrict__ stages,
             const int32_t* __restrict__ cta_first, const typename Fac<T>::acc* __restrict__ vec,
             typename Fac<T>::acc* __restrict__ out, const float* __restrict__ sa, const float* __restrict__ sb,
             int32_t* __restrict__ err) {
  using Acc = typename Fac<T>::acc;
  constexpr int E = Fac<T>::E;
  constexpr int PIECE = kStageBytes / (int)sizeof(T);
  constexpr bool STAGE_VEC = NR == 1;
  extern __shared__ __align__(128) char smem[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
  __shared__ Acc part[2][kConsumerWarps][NR];  // cross-warp partials, double-buffered
  int pbuf = 0;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q0 = cta_first[blockIdx.x], q1 = cta_first[blockIdx.x + 1];
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == 0) {
    produce_segment_stages<T, NR>(F, groups, stages, q0, q1, vec, smem, full, empty, err, lane);
    return;
  }

  // consumers
  const int cw = warp - 1;
  Acc lacc[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) lacc[r] = Acc(0);
  for (int q = q0; q < q1; ++q) {
    const int i = q - q0;
    const int slot = i % kStages;
    if (!mbar_wait(&full[slot], (i / kStages) & 1, err, ERR_WAIT_FULL)) return;
    const char* base = smem + (size_t)slot * kSlotBytes;
    const SlotMeta* meta = reinterpret_cast<const SlotMeta*>(base + kStageBytes + kVecBytes);
    const Stage& st = meta->st;
    if (st.piece < 0) {
      if (st.pad > 0) {
        if constexpr (NR == 1) {
          if (st.last > 0) {
            switch (st.pad * 8 + st.last) {  // (W, KMAX) chosen on the host
#define HD_VB(W, K) case W * 8 + K: consume_vbatch<T, W, K>(meta, base, out, sa, sb, cw, lane); break;
              HD_VB(1, 1) HD_VB(2, 1) HD_VB(2, 2) HD_VB(4, 1) HD_VB(4, 2) HD_VB(4, 4) HD_VB(8, 1) HD_VB(8, 2)
              HD_VB(8, 4) HD_VB(16, 1) HD_VB(16, 2) HD_VB(16, 4) HD_VB(1, 2) HD_VB(1, 4) HD_VB(2, 4)
#undef HD_VB
              default: consume_short<T, NR>(meta, base, vec, out, sa, sb, cw, lane); break;
            }
          } else {
            consume_short<T, NR>(meta, base, vec, out, sa, sb, cw, lane);
          }
        } else {
          consume_short<T, NR>(meta, base, vec, out, sa, sb, cw, lane);
        }
      } else
        consume_long<T, NR>(meta, base, vec, out, sa, sb, cw, lane, &part[0][0][0], pbuf);
    } else {
      // one piece of a long segment: all consumer warps share it; per-lane
      // partials persist across pieces and are combined after the last one
      const SegGroup& G = meta->g[0];
      const int C = st.nelem / E;
      const int64_t vbase = (int64_t)G.vec + (int64_t)st.piece * PIECE;
      for (int c = cw * 32 + lane; c < C; c += kConsumerWarps * 32)
        dot_chunk<T, NR>(base + (size_t)c * 16, vec + (vbase + (int64_t)c * E) * NR, lacc);
      if (st.last) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          Acc a = lacc[r];
          for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
          if (lane == 0) part[pbuf][cw][r] = a;
          lacc[r] = Acc(0);
        }
        consumer_bar();
        if (cw == 0 && lane == 0) {
          Acc tot[NR];
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            tot[r] = Acc(0);
            for (int w = 0; w < kConsumerWarps; ++w) tot[r] += part[pbuf][w][r];
          }
          write_out<T, NR>((int64_t)G.out0 + st.s, tot, out, sa, sb);
        }
        pbuf ^= 1;
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[slot]);
  }
}

// ----------------------------------------------------- U-apply (columns) ----
// y_l(rows of a panel) = sum_k U[:, k] t[tfirst + k]. Threads own fixed row
// chunks of the panel (chunk = 16 bytes of a column) and, when the panel is
// short, one of CG column groups; they stream the panel's columns through the
// same bulk-copy ring and accumulate in registers across stages. No reduction
// is needed except, once per panel, across the CG column groups.
constexpr int kUSlotBytes = kStageBytes + 128;  // factor columns + {Stage, Panel}
struct USlotMeta {
  Stage st;
  Panel P;
};

template <class T, int NR>
__global__ void __launch_bounds__(kSegThreads, 1)
    k_ucols(const T* __restrict__ F, const Panel* __restrict__ panels, const Stage* __restrict__ stages,
            const int32_t* __restrict__ cta_first, const typename Fac<T>::acc* __restrict__ t,
            typename Fac<T>::acc* __restrict__ ylev, int32_t* __restrict__ err) {
  using Acc = typename Fac<T>::acc;
  constexpr int E = Fac<T>::E;
  constexpr int NT = kConsumerWarps * 32;
  extern __shared__ __align__(128) char smem[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
  Acc* red = reinterpret_cast<Acc*>(smem + (size_t)kStages * kUSlotBytes);  // NT * 8

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q0 = cta_first[blockIdx.x], q1 = cta_first[blockIdx.x + 1];
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == 0) {
    if (lane != 0) return;
    int issued = 0;
    bool ok = true;
    for (int q = q0; q < q1; ++q, ++issued) {
      const int slot = issued % kStages;
      const int use = issued / kStages;
      if (use > 0 && !mbar_wait(&empty[slot], (use - 1) & 1, err, ERR_WAIT_EMPTY)) {
        ok = false;
        break;
      }
      char* base = smem + (size_t)slot * kUSlotBytes;
      USlotMeta* meta = reinterpret_cast<USlotMeta*>(base + kStageBytes);
      const Stage st = stages[q];
      meta->st = st;
      meta->P = panels[st.g];
      __threadfence_block();
      const uint32_t bytes = (uint32_t)st.nelem * sizeof(T);
      mbar_expect_tx(&full[slot], bytes);
      bulk_g2s(base, F + st.off, bytes, &full[slot]);
    }
    if (!ok) {
      for (int k = max(0, issued - kStages); k < issued; ++k)
        mbar_wait(&full[k % kStages], (k / kStages) & 1, err, ERR_WAIT_DRAIN);
    }
    return;
  }

  const int ct = (warp - 1) * 32 + lane;
  // FP32 factors: compensated (Kahan) accumulation over the long column loops
  constexpr bool KAHAN = std::is_same<T, float>::value;
  Acc acc[E][NR], cmp[E][NR];
#pragma unroll
  for (int e = 0; e < E; ++e)
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      acc[e][r] = Acc(0);
      cmp[e][r] = Acc(0);
    }
  for (int q = q0; q < q1; ++q) {
    const int i = q - q0;
    const int slot = i % kStages;
    if (!mbar_wait(&full[slot], (i / kStages) & 1, err, ERR_WAIT_FULL)) return;
    const char* base = smem + (size_t)slot * kUSlotBytes;
    const USlotMeta* meta = reinterpret_cast<const USlotMeta*>(base + kStageBytes);
    const Stage st = meta->st;
    const Panel P = meta->P;
    const int RC = P.ld / E;
    int RCP = 1;
    while (RCP < RC) RCP <<= 1;
    const int CG = NT / RCP;
    const int rc = ct % RCP, cg = ct / RCP;
    if (st.ng) {
#pragma unroll
      for (int e = 0; e < E; ++e)
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          acc[e][r] = Acc(0);
          cmp[e][r] = Acc(0);
        }
    }
    if (rc < RC) {
      const Acc* tp = t + ((int64_t)P.tfirst + st.s) * NR;
#pragma unroll 4
      for (int k = cg; k < st.nseg; k += CG) {
        Acc f[E];
        Fac<T>::chunk(base + ((int64_t)k * P.ld + (int64_t)rc * E) * sizeof(T), f);
        Acc tk[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) tk[r] = tp[(int64_t)k * NR + r];
#pragma unroll
        for (int e = 0; e < E; ++e)
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            if constexpr (KAHAN) {
              const Acc y = f[e] * tk[r] - cmp[e][r];
              const Acc s2 = acc[e][r] + y;
              cmp[e][r] = (s2 - acc[e][r]) - y;
              acc[e][r] = s2;
            } else {
              acc[e][r] += f[e] * tk[r];
            }
          }
      }
    }
    if (st.last) {
      if constexpr (KAHAN) {
#pragma unroll
        for (int e = 0; e < E; ++e)
#pragma unroll
          for (int r = 0; r < NR; ++r) acc[e][r] -= cmp[e][r];
      }
      if (CG > 1) {
        // sum the CG column groups, 8 components per pass through `red`
#pragma unroll
        for (int q0c = 0; q0c < E * NR; q0c += 8) {
#pragma unroll
          for (int c = 0; c < 8; ++c)
            if (q0c + c < E * NR) red[(int64_t)ct * 8 + c] = acc[(q0c + c) / NR][(q0c + c) % NR];
          consumer_bar();
          if (cg == 0 && rc < RC) {
            for (int g = 1; g < CG; ++g)
#pragma unroll
              for (int c = 0; c < 8; ++c)
                if (q0c + c < E * NR) acc[(q0c + c) / NR][(q0c + c) % NR] += red[(int64_t)(g * RCP + rc) * 8 + c];
          }
          consumer_bar();
        }
      }
      if (cg == 0 && rc < RC) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int row = rc * E + e;
          if (row < P.R) {
#pragma unroll
            for (int r = 0; r < NR; ++r) ylev[((int64_t)P.out0 + row) * NR + r] = acc[e][r];
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[slot]);
  }
}

// Dynamic shared memory of k_ucols: the ring plus the cross-group reduction buffer.
template <class T, int NR>
constexpr size_t usmem() {
  return (size_t)kStages * kUSlotBytes + (size_t)kConsumerWarps * 32 * 8 * sizeof(typename Fac<T>::acc);
}

// ------------------------------------------------------------- dense ----
// One warp per task (target rows [I0, I0+m) at one level). Rows are handled G
// at a time with 32 / G source stripes. Box-relative FP32 coordinates:
// x_i - x_j = (rel_i - rel_j) + (c_I - c_J) h, where the box offset is exact in
// FP32, so differences keep full FP32 accuracy at the box scale. The FP64 form
// uses the global FP64 coordinates.
template <class Acc, class IO, int NR, int D, bool F64, bool FINAL>
__global__ void __launch_bounds__(256) k_dense(const int4* __restrict__ tasks, int64_t t0, int64_t t1,
                                               const int2* __restrict__ srcs, const float* __restrict__ soff,
                                               const float* __restrict__ rel, const double* __restrict__ p64,
                                               int64_t N, int d_rt, int kid, double kc, double kscale, double kdiag,
                                               const Acc* __restrict__ xt, Acc* __restrict__ ylev_l,
                                               const Acc* __restrict__ ylev, int kappa,
                                               const int32_t* __restrict__ perm, IO* __restrict__ y, int ldy,
                                               int c0) {
  const int d = D > 0 ? D : d_rt;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float kcf = (float)kc;
  for (int64_t it = t0 + warp; it < t1; it += nwarps) {
    const int4 task = tasks[it];
    const int I0 = task.x, m = task.y;
    int G = 1;
    while (G < m && G < 32) G <<= 1;
    const int S = 32 / G;
    const int gi = lane % G, stripe = lane / G;
    for (int g0 = 0; g0 < m; g0 += G) {
      const int row = I0 + g0 + gi;
      const bool valid = g0 + gi < m;
      Acc acc[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[r] = Acc(0);
      if constexpr (F64) {
        double xr[D > 0 ? D : kMaxDim];
        for (int k = 0; k < d; ++k) xr[k] = valid ? p64[(int64_t)k * N + row] : 0.0;
        for (int e = task.z; e < task.w; ++e) {
          const int2 sj = srcs[e];
          for (int j = sj.x + stripe; j < sj.x + sj.y; j += S) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) {
              double t = xr[k] - p64[(int64_t)k * N + j];
              s = fma(t, t, s);
            }
            const double f = f64fast_of_s(kid, s, kc);
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[r] += (Acc)f * xt[(int64_t)j * NR + r];
          }
        }
      } else {
        float xr[D > 0 ? D : kMaxDim];
        for (int k = 0; k < d; ++k) xr[k] = valid ? rel[(int64_t)k * N + row] : 0.f;
        for (int e = task.z; e < task.w; ++e) {
          const int2 sj = srcs[e];
          float off[D > 0 ? D : kMaxDim];
          for (int k = 0; k < d; ++k) off[k] = soff[(int64_t)e * d + k];
          for (int j = sj.x + stripe; j < sj.x + sj.y; j += S) {
            float s = 0.f;
            for (int k = 0; k < d; ++k) {
              float t = (xr[k] - rel[(int64_t)k * N + j]) + off[k];
              s = fmaf(t, t, s);
            }
            const float f = f32_of_s(kid, s, kcf);
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[r] += (Acc)f * xt[(int64_t)j * NR + r];
          }
        }
      }
#pragma unroll
      for (int r = 0; r < NR; ++r)
        for (int o = G; o < 32; o <<= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
      if (stripe == 0 && valid) {
        if constexpr (FINAL) {
          const int64_t orow = perm[row];
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            Acc tot = (Acc)kscale * acc[r] + (Acc)kdiag * xt[(int64_t)row * NR + r];
            for (int l = 1; l <= kappa; ++l) tot += ylev[((int64_t)(l - 1) * N + row) * NR + r];
            y[orow * ldy + c0 + r] = (IO)tot;
          }
        } else {
#pragma unroll
          for (int r = 0; r < NR; ++r) ylev_l[(int64_t)row * NR + r] += (Acc)kscale * acc[r];
        }
      }
    }
  }
}

// Packed near field / dense blocks (FP32, d <= 3, one right-hand side): a
// point is one float4 (box-relative coordinates, x_t in .w); a source box is an
// int4 {J0, n} and its exact box offset; the kernel function is a template
// parameter so the pair loop has no branch on it.
template <int KID>
__device__ __forceinline__ float f32k(float s, float c) {
  if constexpr (KID == HODLRDD_K_LOG) return s == 0.0f ? 0.0f : 0.5f * logf(s);
  else if constexpr (KID == HODLRDD_K_INV_R) return s == 0.0f ? 0.0f : rsqrtf(s);
  else if constexpr (KID == HODLRDD_K_MATERN32) {
    const float a = c * sqrtf(s);
    return (1.0f + a) * expf(-a);
  } else if constexpr (KID == HODLRDD_K_GAUSS) return expf(-c * s);
  else if constexpr (KID == HODLRDD_K_EXP) return expf(-c * sqrtf(s));
  else if constexpr (KID == HODLRDD_K_INV_R2_4D) return s == 0.0f ? 0.0f : c / s;
  else if constexpr (KID == HODLRDD_K_R) return sqrtf(s);
  else if constexpr (KID == HODLRDD_K_SIN) return sinf(sqrtf(s));
  else return rsqrtf(1.0f + sqrtf(s));
}

template <int D, int KID, bool FINAL>
__global__ void __launch_bounds__(256) k_dense4(const int4* __restrict__ tasks, int64_t t0, int64_t t1,
                                                const int4* __restrict__ srcs, const float4* __restrict__ soff,
                                                const float4* __restrict__ P, int64_t N, float kc, float kscale,
                                                float kdiag, float* __restrict__ ylev_l,
                                                const float* __restrict__ ylev, int kappa,
                                                const int32_t* __restrict__ perm, float* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it = t0 + warp; it < t1; it += nwarps) {
    const int4 task = tasks[it];
    const int I0 = task.x, m = task.y;
    int G = 1;
    while (G < m && G < 32) G <<= 1;
    const int S = 32 / G;
    const int gi = lane % G, stripe = lane / G;
    for (int g0 = 0; g0 < m; g0 += G) {
      const int row = I0 + g0 + gi;
      const bool valid = g0 + gi < m;
      const float4 xr = valid ? P[row] : make_float4(0.f, 0.f, 0.f, 0.f);
      float acc0 = 0.f, acc1 = 0.f;
      for (int e = task.z; e < task.w; ++e) {
        const int4 sj = srcs[e];
        const float4 of = soff[e];
        const int j1 = sj.x + sj.y;
        int j = sj.x + stripe;
        for (; j + S < j1; j += 2 * S) {  // two independent pairs in flight
          const float4 p0 = P[j], p1 = P[j + S];
          float s0 = 0.f, s1 = 0.f, t;
          t = (xr.x - p0.x) + of.x; s0 = fmaf(t, t, s0);
          t = (xr.x - p1.x) + of.x; s1 = fmaf(t, t, s1);
          if (D > 1) {
            t = (xr.y - p0.y) + of.y; s0 = fmaf(t, t, s0);
            t = (xr.y - p1.y) + of.y; s1 = fmaf(t, t, s1);
          }
          if (D > 2) {
            t = (xr.z - p0.z) + of.z; s0 = fmaf(t, t, s0);
            t = (xr.z - p1.z) + of.z; s1 = fmaf(t, t, s1);
          }
          acc0 = fmaf(f32k<KID>(s0, kc), p0.w, acc0);
          acc1 = fmaf(f32k<KID>(s1, kc), p1.w, acc1);
        }
        if (j < j1) {
          const float4 p0 = P[j];
          float s0 = 0.f, t;
          t = (xr.x - p0.x) + of.x; s0 = fmaf(t, t, s0);
          if (D > 1) { t = (xr.y - p0.y) + of.y; s0 = fmaf(t, t, s0); }
          if (D > 2) { t = (xr.z - p0.z) + of.z; s0 = fmaf(t, t, s0); }
          acc0 = fmaf(f32k<KID>(s0, kc), p0.w, acc0);
        }
      }
      float acc = acc0 + acc1;
      for (int o = G; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (stripe == 0 && valid) {
        if constexpr (FINAL) {
          float tot = kscale * acc + kdiag * xr.w;
          for (int l = 1; l <= kappa; ++l) tot += ylev[(int64_t)(l - 1) * N + row];
          y[perm[row]] = tot;
        } else {
          ylev_l[row] += kscale * acc;
        }
      }
    }
  }
}

// One right-hand side with packed points: x_t[i] and the .w lane of every
// packed level array.
template <class IO>
__global__ void k_gather_pack(const IO* __restrict__ x, const int32_t* __restrict__ perm, int64_t N, int ldx,
                              int c0, float* __restrict__ xt, float4* const* __restrict__ packs, int npacks) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = (float)x[(int64_t)perm[i] * ldx + c0];
    xt[i] = v;
    for (int k = 0; k < npacks; ++k) packs[k][i].w = v;
  }
}

__global__ void k_pack_rel4(const float* __restrict__ rel, int64_t N, int d, float4* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = make_float4(rel[i], d > 1 ? rel[N + i] : 0.f, d > 2 ? rel[2 * N + i] : 0.f, 0.f);
}

template <class Acc, class IO, int NR>
__global__ void k_gather(const IO* __restrict__ x, const int32_t* __restrict__ perm, int64_t N, int ldx, int c0,
                         Acc* __restrict__ xt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const IO* src = x + (int64_t)perm[i] * ldx + c0;
#pragma unroll
    for (int r = 0; r < NR; ++r) xt[i * NR + r] = (Acc)src[r];
  }
}

// ---------------------------------------------------------------- packing ----
// Column source offsets in the FP64 ACA output: colU[c] / colV[c] for global
// column c = toff[b] + k.
__global__ void k_colmap(int64_t nblk, const int32_t* __restrict__ rank, const int32_t* __restrict__ bm,
                         const int32_t* __restrict__ bn, const int64_t* __restrict__ toff,
                         const int64_t* __restrict__ uoff64, const int64_t* __restrict__ voff64,
                         int64_t* __restrict__ colU, int64_t* __restrict__ colV) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < rank[b]; ++k) {
      colU[toff[b] + k] = uoff64[b] + (int64_t)k * bm[b];
      colV[toff[b] + k] = voff64[b] + (int64_t)k * bn[b];
    }
}

// One warp per column: power-of-two scale >= max |entry| (16-bit), else 1.
__global__ void k_colscale(int64_t ncol, const int64_t* __restrict__ colU, const int64_t* __restrict__ colV,
                           const int32_t* __restrict__ colrows_u, const int32_t* __restrict__ colrows_v,
                           const double* __restrict__ U64, const double* __restrict__ V64, int scaled,
                           float* __restrict__ su, float* __restrict__ sv) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = warp; c < ncol; c += nw) {
    for (int side = 0; side < 2; ++side) {
      const double* col = side == 0 ? U64 + colU[c] : V64 + colV[c];
      const int rows = side == 0 ? colrows_u[c] : colrows_v[c];
      double mx = 0.0;
      if (scaled)
        for (int i = lane; i < rows; i += 32) mx = fmax(mx, fabs(col[i]));
      for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      int e = 0;
      if (mx > 0.0) frexp(mx, &e);
      const float sc = mx > 0.0 ? (float)ldexp(1.0, e) : 1.0f;
      if (lane == 0) (side == 0 ? su : sv)[c] = sc;
    }
  }
}

// V stream: one CTA per group (= block); segment k = column k, lead pad a.
template <class T>
__global__ void k_packV(int64_t ngroups, const SegGroup* __restrict__ groups, const int32_t* __restrict__ lead,
                        const int32_t* __restrict__ nrows, const int64_t* __restrict__ colV,
                        const double* __restrict__ V64, const float* __restrict__ sv, T* __restrict__ out) {
  for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
    const SegGroup G = groups[g];
    const int a = lead[g], n = nrows[g];
    for (int k = 0; k < G.cnt; ++k) {
      const int64_t c = (int64_t)G.out0 + k;
      const double* col = V64 + colV[c];
      const double inv = 1.0 / (double)sv[c];
      T* dst = out + G.off + (int64_t)k * G.L;
      for (int e = threadIdx.x; e < G.L; e += blockDim.x)
        dst[e] = Fac<T>::from((e >= a && e < a + n) ? col[e - a] * inv : 0.0);
    }
  }
}

// U stream: one CTA per panel; element (r, k) of the column-major panel is row
// r0 + r of global column tfirst + k, divided by its scale (zero below R).
template <class T>
__global__ void k_packU(int64_t npanels, const Panel* __restrict__ panels, const int32_t* __restrict__ prow0,
                        const int64_t* __restrict__ colU, const double* __restrict__ U64,
                        const float* __restrict__ su, T* __restrict__ out) {
  for (int64_t p = blockIdx.x; p < npanels; p += gridDim.x) {
    const Panel Pn = panels[p];
    const int r0 = prow0[p];
    for (int64_t idx = threadIdx.x; idx < (int64_t)Pn.P * Pn.ld; idx += blockDim.x) {
      const int k = (int)(idx / Pn.ld), r = (int)(idx % Pn.ld);
      const int64_t c = (int64_t)Pn.tfirst + k;
      const double v = r < Pn.R ? U64[colU[c] + r0 + r] / (double)su[c] : 0.0;
      out[Pn.off + idx] = Fac<T>::from(v);
    }
  }
}

// Box-relative FP32 coordinates at level l: rel = x - (lo + c_box * h).
__global__ void k_relcoords(const double* __restrict__ p64, int64_t N, int d, int l,
                            const int32_t* __restrict__ bstart, const uint64_t* __restrict__ bkey, int64_t nb,
                            const double* __restrict__ lo, double h, float* __restrict__ rel) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t a = 0, b = nb;  // last box with bstart <= i
    while (b - a > 1) {
      int64_t mid = (a + b) >> 1;
      if (bstart[mid] <= i) a = mid; else b = mid;
    }
    const uint64_t key = bkey[a];
    for (int k = 0; k < d; ++k) {
      int64_t c = 0;
      for (int bit = 0; bit < l; ++bit) c |= (int64_t)((key >> (d * bit + k)) & 1u) << bit;
      rel[(int64_t)k * N + i] = (float)(p64[(int64_t)k * N + i] - (lo[k] + (double)c * h));
    }
  }
}

int grid_warps(int64_t items, int sms) {
  int64_t ctas = (items + 7) / 8;
  int64_t cap = (int64_t)sms * 8;
  if (ctas > cap) ctas = cap;
  if (ctas < 1) ctas = 1;
  return (int)ctas;
}

// Stage schedule of a stream: whole segments packed into stages of at most
// kStageBytes; segments longer than a stage become pieces. CTA ranges are
// balanced by bytes and never cut a long segment.
void schedule(Stream& S, size_t esize, size_t vsize, int E, int ctas) {
  const int64_t cap = kStageBytes / (int64_t)esize;
  S.h_stages.clear();
  Stage cur{0, 0, -1, 0, 0, -1, 0, 0, 0};
  int64_t cur_vbytes = 0, cur_group = -1, cur_maxc = 0;
  auto flush = [&]() {
    if (cur.nseg > 0) {
      if (cur.pad != 0) {
        if (cur_maxc < kBatchChunks) {
          // batched: W lanes own up to KMAX = 4 chunks each (W, KMAX powers of two)
          int64_t w = 1;
          while (w * 4 < cur_maxc) w <<= 1;
          int64_t k = 1;
          while (w * k < cur_maxc) k <<= 1;
          cur.pad = (int32_t)w;
          cur.last = (int32_t)k;
        } else {
          // one team of TS lanes per segment
          int ts = 1;
          while (ts < cur_maxc && ts < 32) ts <<= 1;
          cur.pad = ts;
          cur.last = 0;
        }
      }
      S.h_stages.push_back(cur);
    }
    cur = Stage{0, 0, -1, 0, 0, -1, 0, 0, 0};
    cur_vbytes = 0;
    cur_group = -1;
    cur_maxc = 0;
  };
  for (int64_t g = 0; g < (int64_t)S.h_groups.size(); ++g) {
    const SegGroup& G = S.h_groups[g];
    const int64_t C = G.L / E;
    if (G.L > cap) {  // pieces
      flush();
      for (int s = 0; s < G.cnt; ++s)
        for (int64_t p0 = 0, piece = 0; p0 < G.L; p0 += cap, ++piece) {
          const int64_t len = std::min<int64_t>(cap, G.L - p0);
          S.h_stages.push_back(Stage{G.off + (int64_t)s * G.L + p0, (int32_t)len, (int32_t)g, s, 0,
                                     (int32_t)piece, p0 + len >= G.L ? 1 : 0, 1, 0});
        }
      continue;
    }
    if (C > kLongChunks) {  // long stages: whole segments of this group only
      flush();
      for (int s = 0; s < G.cnt; ++s) {
        if (cur.nseg > 0 && cur.nelem + G.L > cap) flush();
        if (cur.nseg == 0) cur = Stage{G.off + (int64_t)s * G.L, 0, (int32_t)g, s, 0, -1, 0, 1, 0};
        cur.nelem += G.L;
        cur.nseg += 1;
      }
      flush();
      continue;
    }
    const int64_t vb = G.L * (int64_t)vsize <= kVecBytes ? G.L * (int64_t)vsize : 0;
    for (int s = 0; s < G.cnt; ++s) {
      const bool new_group = cur_group != g;
      if (cur.nseg > 0 &&
          (cur.nelem + G.L > cap || (new_group && (cur.ng + 1 > kGmax || cur_vbytes + vb > kVecBytes))))
        flush();
      if (cur.nseg == 0) {
        cur.off = G.off + (int64_t)s * G.L;
        cur.g = (int32_t)g;
        cur.s = s;
        cur.pad = 1;  // marks a short stage; the team size is set at flush
      }
      if (cur_group != g) {
        cur.ng += 1;
        cur_vbytes += vb;
        cur_group = g;
        cur_maxc = std::max(cur_maxc, C);
      }
      cur.nelem += G.L;
      cur.nseg += 1;
    }
  }
  flush();
  // balance CTAs by bytes, cutting only between whole segments
  int64_t total = 0;
  for (const Stage& st : S.h_stages) total += st.nelem;
  S.h_cta.assign(1, 0);
  int64_t acc = 0;
  const int64_t target = std::max<int64_t>(1, (total + ctas - 1) / ctas);
  for (size_t q = 0; q < S.h_stages.size(); ++q) {
    acc += S.h_stages[q].nelem;
    const bool cut_ok = S.h_stages[q].piece < 0 || S.h_stages[q].last;
    if (cut_ok && acc >= target * (int64_t)S.h_cta.size() && (int)S.h_cta.size() < ctas)
      S.h_cta.push_back((int32_t)(q + 1));
  }
  if (S.h_cta.back() != (int32_t)S.h_stages.size()) S.h_cta.push_back((int32_t)S.h_stages.size());
  S.ctas = (int)S.h_cta.size() - 1;
}

// Stage schedule of the U panels: whole columns of one panel per stage; CTA
// ranges are balanced by bytes and cut only at panel boundaries.
void schedule_panels(Stream& S, size_t esize, int ctas) {
  S.h_stages.clear();
  for (int64_t p = 0; p < (int64_t)S.h_panels.size(); ++p) {
    const Panel& Pn = S.h_panels[p];
    const int per = std::max<int>(1, (int)(kStageBytes / ((int64_t)Pn.ld * (int64_t)esize)));
    for (int k0 = 0; k0 < Pn.P; k0 += per) {
      const int nc = std::min(per, Pn.P - k0);
      S.h_stages.push_back(Stage{Pn.off + (int64_t)k0 * Pn.ld, (int32_t)((int64_t)nc * Pn.ld), (int32_t)p, k0, nc,
                                 -1, k0 + nc >= Pn.P ? 1 : 0, k0 == 0 ? 1 : 0, 0});
    }
  }
  int64_t total = 0;
  for (const Stage& st : S.h_stages) total += st.nelem;
  S.h_cta.assign(1, 0);
  int64_t acc = 0;
  const int64_t target = std::max<int64_t>(1, (total + ctas - 1) / ctas);
  for (size_t q = 0; q < S.h_stages.size(); ++q) {
    acc += S.h_stages[q].nelem;
    if (S.h_stages[q].last && acc >= target * (int64_t)S.h_cta.size() && (int)S.h_cta.size() < ctas)
      S.h_cta.push_back((int32_t)(q + 1));
  }
  if (S.h_cta.back() != (int32_t)S.h_stages.size()) S.h_cta.push_back((int32_t)S.h_stages.size());
  S.ctas = (int)S.h_cta.size() - 1;
}

template <class T>
int pack_typed(hodlrdd_s* h, const DevBuf<double>& U64, const DevBuf<double>& V64,
               const std::vector<int64_t>& uoff64, const std::vector<int64_t>& voff64) {
  cudaStream_t st = h->st;
  using Acc = typename Fac<T>::acc;
  constexpr int E = Fac<T>::E;
  const int A1 = 16 / (int)sizeof(Acc);  // vector alignment in elements
  const int64_t nblk = h->nblk;
  Plan& P = h->plan;
  auto roundE = [&](int64_t v) { return (v + E - 1) / E * E; };
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);

  // V groups: one per low-rank block
  P.vs.h_groups.clear();
  P.h_vgroup.assign(nblk, -1);
  std::vector<int32_t> vlead, vrows;
  int64_t off = 0;
  for (int64_t b = 0; b < nblk; ++b) {
    const int p = h->h_rank[b];
    if (p == 0) continue;
    const int a = (int)(h->h_bJ0[b] % A1);
    const int64_t L = roundE(a + h->h_bn[b]);
    P.h_vgroup[b] = (int64_t)P.vs.h_groups.size();
    P.vs.h_groups.push_back(SegGroup{off, (int32_t)L, p, h->h_bJ0[b] - a, (int32_t)h->h_toff[b]});
    vlead.push_back(a);
    vrows.push_back(h->h_bn[b]);
    off += L * p;
  }
  P.vs.elems = off;
  // U panels: per (level, box) with low-rank blocks, rows in panels of at most
  // kPanelRows, column-major over the box's concatenated IL columns
  P.us.h_panels.clear();
  P.h_ugroup.assign(nblk, -1);
  P.h_ucol.assign(nblk, 0);
  std::vector<int32_t> prow0;
  off = 0;
  for (int l = 1; l <= h->kappa; ++l) {
    const Level& L = h->lv[l];
    for (int64_t i = 0; i < L.nb; ++i) {
      const int64_t b0 = h->h_blk_off[l] + L.h_iloff[i], b1 = h->h_blk_off[l] + L.h_iloff[i + 1];
      int64_t Pi = 0, tf = -1;
      for (int64_t b = b0; b < b1; ++b)
        if (h->h_rank[b] > 0) {
          if (tf < 0) tf = h->h_toff[b];
          P.h_ugroup[b] = (int64_t)P.us.h_panels.size();
          P.h_ucol[b] = (int32_t)Pi;
          Pi += h->h_rank[b];
        }
      if (Pi == 0) continue;
      const int32_t I0 = L.h_bstart[i], m = L.h_bstart[i + 1] - I0;
      for (int32_t r0 = 0; r0 < m; r0 += kPanelRows) {
        const int32_t R = std::min(kPanelRows, m - r0);
        const int64_t ld = roundE(R);
        P.us.h_panels.push_back(Panel{off, (int32_t)ld, R, (int32_t)Pi, (int32_t)tf,
                                      (int32_t)((int64_t)(l - 1) * h->N + I0 + r0), 0});
        prow0.push_back(r0);
        off += ld * Pi;
      }
    }
  }
  P.us.elems = off;
  if ((int64_t)h->total_rank + 2 * kGuard >= INT32_MAX || (int64_t)h->kappa * h->N >= INT32_MAX) {
    set_error("problem too large for 32-bit vector indices");
    return HODLRDD_ERR_UNSUPPORTED;
  }
  schedule(P.vs, sizeof(T), sizeof(Acc), E, sms);
  schedule_panels(P.us, sizeof(T), sms);

  // column maps, scales, packing
  const int64_t ncol = h->total_rank;
  DevBuf<int64_t> colU, colV, du64, dv64;
  DevBuf<int32_t> crows_u, crows_v, dvlead, dvrows, dprow0;
  std::vector<int32_t> hcru(std::max<int64_t>(ncol, 1)), hcrv(std::max<int64_t>(ncol, 1));
  for (int64_t b = 0; b < nblk; ++b)
    for (int k = 0; k < h->h_rank[b]; ++k) {
      hcru[h->h_toff[b] + k] = h->h_bm[b];
      hcrv[h->h_toff[b] + k] = h->h_bn[b];
    }
  HD_TRY(colU.alloc(std::max<int64_t>(ncol, 1)));
  HD_TRY(colV.alloc(std::max<int64_t>(ncol, 1)));
  HD_TRY(upload(du64, uoff64, st));
  HD_TRY(upload(dv64, voff64, st));
  HD_TRY(upload(crows_u, hcru, st));
  HD_TRY(upload(crows_v, hcrv, st));
  HD_TRY(upload(dvlead, vlead, st));
  HD_TRY(upload(dvrows, vrows, st));
  HD_TRY(upload(dprow0, prow0, st));
  HD_TRY(h->su.alloc(std::max<int64_t>(ncol, 1)));
  HD_TRY(h->sv.alloc(std::max<int64_t>(ncol, 1)));
  HD_TRY(P.vs.data.alloc((size_t)std::max<int64_t>(P.vs.elems, E) * sizeof(T)));
  HD_TRY(P.us.data.alloc((size_t)std::max<int64_t>(P.us.elems, E) * sizeof(T)));
  HD_TRY(upload(P.vs.groups, P.vs.h_groups, st));
  HD_TRY(upload(P.us.panels, P.us.h_panels, st));
  HD_TRY(upload(P.vs.stages, P.vs.h_stages, st));
  HD_TRY(upload(P.us.stages, P.us.h_stages, st));
  HD_TRY(upload(P.vs.cta, P.vs.h_cta, st));
  HD_TRY(upload(P.us.cta, P.us.h_cta, st));
  if (ncol > 0) {
    k_colmap<<<(int)std::min<int64_t>((nblk + 255) / 256, 4096), 256, 0, st>>>(
        nblk, h->rank.p, h->bm.p, h->bn.p, h->toff.p, du64.p, dv64.p, colU.p, colV.p);
    k_colscale<<<grid_warps(ncol, sms), 256, 0, st>>>(ncol, colU.p, colV.p, crows_u.p, crows_v.p, U64.p, V64.p,
                                                      Fac<T>::scaled ? 1 : 0, h->su.p, h->sv.p);
    const int64_t nvg = (int64_t)P.vs.h_groups.size(), nup = (int64_t)P.us.h_panels.size();
    if (nvg)
      k_packV<T><<<(int)std::min<int64_t>(nvg, sms * 16), 256, 0, st>>>(
          nvg, P.vs.groups.p, dvlead.p, dvrows.p, colV.p, V64.p, h->sv.p, reinterpret_cast<T*>(P.vs.data.p));
    if (nup)
      k_packU<T><<<(int)std::min<int64_t>(nup, sms * 16), 256, 0, st>>>(nup, P.us.panels.p, dprow0.p, colU.p, U64.p,
                                                                        h->su.p, reinterpret_cast<T*>(P.us.data.p));
    HD_CUDA(cudaGetLastError());
  }
  HD_CUDA(cudaStreamSynchronize(st));
  h->factor_bytes = (P.vs.elems + P.us.elems) * (int64_t)sizeof(T) + (Fac<T>::scaled ? 2 * ncol * 4 : 0);
  return HODLRDD_OK;
}

}  // namespace

int pack_factors(hodlrdd_s* h, const DevBuf<double>& U64, const DevBuf<double>& V64,
                 const std::vector<int64_t>& uoff64, const std::vector<int64_t>& voff64) {
  h->h_toff.assign(h->nblk + 1, 0);
  h->factor_elems = 0;
  for (int64_t b = 0; b < h->nblk; ++b) {
    h->h_toff[b + 1] = h->h_toff[b] + h->h_rank[b];
    h->factor_elems += (int64_t)h->h_rank[b] * (h->h_bm[b] + h->h_bn[b]);
  }
  switch (h->opt.precision) {
    case HODLRDD_PREC_FP64: return pack_typed<double>(h, U64, V64, uoff64, voff64);
    case HODLRDD_PREC_FP32: return pack_typed<float>(h, U64, V64, uoff64, voff64);
    case HODLRDD_PREC_FP16: return pack_typed<__half>(h, U64, V64, uoff64, voff64);
    default: return pack_typed<__nv_bfloat16>(h, U64, V64, uoff64, voff64);
  }
}

// Dense task lists (near field and dense-flagged IL blocks) and the per-level
// box-relative coordinates they read.
int build_plan(hodlrdd_s* h) {
  Plan& P = h->plan;
  const int d = h->d;
  const bool f64 = h->opt.precision == HODLRDD_PREC_FP64;
  std::vector<int4> tasks;
  std::vector<int2> srcs;
  std::vector<float> soff;
  // reference side of level-l boxes rounded to 20 significant bits, so that
  // (c_I - c_J) h is exact in FP32 for |c_I - c_J| < 16
  P.h_box.assign(h->kappa + 1, 0.0);
  for (int l = 0; l <= h->kappa; ++l) {
    int e = 0;
    double m = std::frexp(std::ldexp(h->side, -l), &e);
    P.h_box[l] = std::ldexp(std::nearbyint(std::ldexp(m, 20)), e - 20);
  }
  auto coords = [&](int l, int64_t b, int64_t* c) {
    const uint64_t key = h->lv[l].h_bkey[b];
    for (int k = 0; k < d; ++k) {
      c[k] = 0;
      for (int bit = 0; bit < l; ++bit) c[k] |= (int64_t)((key >> (d * bit + k)) & 1u) << bit;
    }
  };
  auto add_src = [&](int l, int64_t I, int64_t J) {
    const Level& L = h->lv[l];
    srcs.push_back(make_int2(L.h_bstart[J], L.h_bstart[J + 1] - L.h_bstart[J]));
    int64_t cI[kMaxDim], cJ[kMaxDim];
    coords(l, I, cI);
    coords(l, J, cJ);
    for (int k = 0; k < d; ++k) soff.push_back((float)((double)(cI[k] - cJ[k]) * P.h_box[l]));
  };
  h->dense_pairs = 0;
  P.coarse.clear();
  std::vector<char> need_rel(h->kappa + 1, 0);
  for (int l = 1; l < h->kappa; ++l) {
    const Level& L = h->lv[l];
    DenseLevel DL;
    DL.level = l;
    DL.t0 = (int64_t)tasks.size();
    for (int64_t i = 0; i < L.nb; ++i) {
      const int64_t b0 = h->h_blk_off[l] + L.h_iloff[i], b1 = h->h_blk_off[l] + L.h_iloff[i + 1];
      const int32_t s0 = (int32_t)srcs.size();
      for (int64_t b = b0; b < b1; ++b)
        if (h->h_dense[b]) {
          add_src(l, i, h->h_bsj[b]);
          h->dense_pairs += (int64_t)h->h_bm[b] * h->h_bn[b];
        }
      const int32_t s1 = (int32_t)srcs.size();
      if (s1 == s0) continue;
      const int32_t I0 = L.h_bstart[i], m = L.h_bstart[i + 1] - I0;
      for (int32_t r = 0; r < m; r += 32) tasks.push_back(make_int4(I0 + r, std::min(32, m - r), s0, s1));
    }
    DL.t1 = (int64_t)tasks.size();
    if (DL.t1 > DL.t0) {
      P.coarse.push_back(DL);
      need_rel[l] = 1;
    }
  }
  {
    const int l = h->kappa;
    const Level& L = h->lv[l];
    P.leaf.level = l;
    P.leaf.t0 = (int64_t)tasks.size();
    for (int64_t i = 0; i < L.nb; ++i) {
      const int32_t s0 = (int32_t)srcs.size();
      const int32_t I0 = L.h_bstart[i], m = L.h_bstart[i + 1] - I0;
      for (int32_t e = h->h_nearoff[i]; e < h->h_nearoff[i + 1]; ++e) {
        add_src(l, i, h->h_nearidx[e]);
        h->dense_pairs += (int64_t)m * srcs.back().y;
      }
      if (l >= 1) {
        const int64_t b0 = h->h_blk_off[l] + L.h_iloff[i], b1 = h->h_blk_off[l] + L.h_iloff[i + 1];
        for (int64_t b = b0; b < b1; ++b)
          if (h->h_dense[b]) {
            add_src(l, i, h->h_bsj[b]);
            h->dense_pairs += (int64_t)m * h->h_bn[b];
          }
      }
      tasks.push_back(make_int4(I0, m, s0, (int32_t)srcs.size()));
    }
    P.leaf.t1 = (int64_t)tasks.size();
    need_rel[l] = 1;
  }
  if ((int64_t)srcs.size() >= INT32_MAX) {
    set_error("dense source list too long");
    return HODLRDD_ERR_UNSUPPORTED;
  }
  cudaStream_t st = h->st;
  HD_TRY(upload(P.tasks, tasks, st));
  HD_TRY(upload(P.srcs, srcs, st));
  HD_TRY(upload(P.soff, soff, st));
  P.rel.clear();
  P.rel.resize(h->kappa + 1);
  if (!f64) {
    std::vector<double> hlo(h->lo, h->lo + d);
    DevBuf<double> dlo;
    HD_TRY(upload(dlo, hlo, st));
    for (int l = 0; l <= h->kappa; ++l) {
      if (!need_rel[l]) continue;
      HD_TRY(P.rel[l].alloc((size_t)h->N * d));
      const Level& L = h->lv[l];
      k_relcoords<<<(int)std::min<int64_t>((h->N + 255) / 256, 152 * 16), 256, 0, st>>>(
          h->pts64.p, h->N, d, l, L.bstart.p, L.bkey.p, L.nb, dlo.p, P.h_box[l], P.rel[l].p);
      HD_CUDA(cudaGetLastError());
    }
    if (d <= 3) {
      P.rel4.clear();
      P.rel4.resize(h->kappa + 1);
      std::vector<int32_t> lvls;
      std::vector<float4*> ptrs;
      for (int l = 0; l <= h->kappa; ++l) {
        if (!need_rel[l]) continue;
        HD_TRY(P.rel4[l].alloc(h->N));
        k_pack_rel4<<<(int)std::min<int64_t>((h->N + 255) / 256, 152 * 16), 256, 0, st>>>(P.rel[l].p, h->N, d,
                                                                                         P.rel4[l].p);
        HD_CUDA(cudaGetLastError());
        lvls.push_back(l);
        ptrs.push_back(P.rel4[l].p);
      }
      HD_TRY(upload(P.rel4_levels, lvls, st));
      HD_TRY(upload(P.rel4_ptrs, ptrs, st));
      std::vector<int4> s4(srcs.size());
      std::vector<float4> o4(srcs.size());
      for (size_t e = 0; e < srcs.size(); ++e) {
        s4[e] = make_int4(srcs[e].x, srcs[e].y, 0, 0);
        o4[e] = make_float4(soff[e * d], d > 1 ? soff[e * d + 1] : 0.f, d > 2 ? soff[e * d + 2] : 0.f, 0.f);
      }
      HD_TRY(upload(P.srcs4, s4, st));
      HD_TRY(upload(P.soff4, o4, st));
    }
    HD_CUDA(cudaStreamSynchronize(st));
  }
  HD_CUDA(cudaStreamSynchronize(st));
  return HODLRDD_OK;
}

int alloc_workspace(hodlrdd_s* h) {
  const int nr = 8;
  const size_t acc = h->opt.precision == HODLRDD_PREC_FP64 ? 8 : 4;
  HD_TRY(h->xt.alloc(((size_t)h->N + 2 * kGuard) * nr * acc));
  HD_TRY(h->tbuf.alloc(((size_t)h->total_rank + 2 * kGuard) * nr * acc));
  HD_TRY(h->ylev.alloc((size_t)std::max(h->kappa, 1) * h->N * nr * acc));
  HD_TRY(h->err.alloc(1));
  HD_CUDA(cudaMemsetAsync(h->xt.p, 0, h->xt.bytes(), h->st));
  HD_CUDA(cudaMemsetAsync(h->tbuf.p, 0, h->tbuf.bytes(), h->st));
  HD_CUDA(cudaMemsetAsync(h->err.p, 0, sizeof(int32_t), h->st));
  HD_CUDA(cudaStreamSynchronize(h->st));
  return HODLRDD_OK;
}

namespace {

// Tracing: take 5 events for one chunk from the handle's pool.
int chunk_events(hodlrdd_s* h, cudaEvent_t* ev) {
  for (int i = 0; i < 5; ++i) {
    if (h->ev_pool.empty()) {
      cudaEvent_t e;
      HD_CUDA(cudaEventCreate(&e));
      h->ev_pool.push_back(e);
    }
    ev[i] = h->ev_pool.back();
    h->ev_pool.pop_back();
  }
  h->ev_pending.emplace_back(ev, ev + 5);
  return HODLRDD_OK;
}

template <class Acc, class IO, int NR, int D, bool F64>
int launch_dense(hodlrdd_s* h, cudaStream_t st, int sms, const Acc* xt, Acc* yl, IO* y, int ldy, int c0) {
  const Plan& P = h->plan;
  const double kc = kernel_const(h->K);
  for (const DenseLevel& DL : P.coarse) {
    const float* rel = F64 ? nullptr : P.rel[DL.level].p;
    k_dense<Acc, IO, NR, D, F64, false><<<grid_warps(DL.t1 - DL.t0, sms), 256, 0, st>>>(
        P.tasks.p, DL.t0, DL.t1, P.srcs.p, P.soff.p, rel, h->pts64.p, h->N, h->d, h->K.id, kc, h->K.scale,
        h->K.diag, xt, yl + (int64_t)(DL.level - 1) * h->N * NR, yl, h->kappa, h->perm.p, y, ldy, c0);
    h->launches += 1;
  }
  const float* rel = F64 ? nullptr : P.rel[h->kappa].p;
  k_dense<Acc, IO, NR, D, F64, true><<<grid_warps(P.leaf.t1 - P.leaf.t0, sms), 256, 0, st>>>(
      P.tasks.p, P.leaf.t0, P.leaf.t1, P.srcs.p, P.soff.p, rel, h->pts64.p, h->N, h->d, h->K.id, kc, h->K.scale,
      h->K.diag, xt, nullptr, yl, h->kappa, h->perm.p, y, ldy, c0);
  h->launches += 1;
  HD_CUDA(cudaGetLastError());
  return HODLRDD_OK;
}

template <int D, int KID>
void launch_dense4_k(hodlrdd_s* h, cudaStream_t st, int sms, float* yl, float* y) {
  const Plan& P = h->plan;
  const float kc = (float)kernel_const(h->K);
  for (const DenseLevel& DL : P.coarse) {
    k_dense4<D, KID, false><<<grid_warps(DL.t1 - DL.t0, sms), 256, 0, st>>>(
        P.tasks.p, DL.t0, DL.t1, P.srcs4.p, P.soff4.p, P.rel4[DL.level].p, h->N, kc, (float)h->K.scale,
        (float)h->K.diag, yl + (int64_t)(DL.level - 1) * h->N, yl, h->kappa, h->perm.p, y);
    h->launches += 1;
  }
  k_dense4<D, KID, true><<<grid_warps(P.leaf.t1 - P.leaf.t0, sms), 256, 0, st>>>(
      P.tasks.p, P.leaf.t0, P.leaf.t1, P.srcs4.p, P.soff4.p, P.rel4[h->kappa].p, h->N, kc, (float)h->K.scale,
      (float)h->K.diag, nullptr, yl, h->kappa, h->perm.p, y);
  h->launches += 1;
}

template <int D>
void launch_dense4_d(hodlrdd_s* h, cudaStream_t st, int sms, float* yl, float* y) {
  switch (h->K.id) {
    case HODLRDD_K_LOG: launch_dense4_k<D, HODLRDD_K_LOG>(h, st, sms, yl, y); break;
    case HODLRDD_K_INV_R: launch_dense4_k<D, HODLRDD_K_INV_R>(h, st, sms, yl, y); break;
    case HODLRDD_K_MATERN32: launch_dense4_k<D, HODLRDD_K_MATERN32>(h, st, sms, yl, y); break;
    case HODLRDD_K_GAUSS: launch_dense4_k<D, HODLRDD_K_GAUSS>(h, st, sms, yl, y); break;
    case HODLRDD_K_EXP: launch_dense4_k<D, HODLRDD_K_EXP>(h, st, sms, yl, y); break;
    case HODLRDD_K_INV_R2_4D: launch_dense4_k<D, HODLRDD_K_INV_R2_4D>(h, st, sms, yl, y); break;
    case HODLRDD_K_R: launch_dense4_k<D, HODLRDD_K_R>(h, st, sms, yl, y); break;
    case HODLRDD_K_SIN: launch_dense4_k<D, HODLRDD_K_SIN>(h, st, sms, yl, y); break;
    default: launch_dense4_k<D, HODLRDD_K_INV_SQRT1P>(h, st, sms, yl, y); break;
  }
}

// Packed dense / near-field launches (FP32, d <= 3, one right-hand side, y of
// type float with leading dimension 1).
template <class IO>
int launch_dense4(hodlrdd_s* h, cudaStream_t st, int sms, float* yl, IO* y, int ldy, int c0) {
  if constexpr (!std::is_same<IO, float>::value) {
    set_error("packed near field needs float output");
    return HODLRDD_ERR_UNSUPPORTED;
  } else {
    if (ldy != 1 || c0 != 0) {
      set_error("packed near field is for one right-hand side");
      return HODLRDD_ERR_UNSUPPORTED;
    }
    switch (h->d) {
      case 1: launch_dense4_d<1>(h, st, sms, yl, y); break;
      case 2: launch_dense4_d<2>(h, st, sms, yl, y); break;
      default: launch_dense4_d<3>(h, st, sms, yl, y); break;
    }
    HD_CUDA(cudaGetLastError());
    return HODLRDD_OK;
  }
}

template <class T, class IO, int NR>
int matvec_chunk(hodlrdd_s* h, const IO* x, IO* y, int ldx, int c0, cudaStream_t st) {
  using Acc = typename Fac<T>::acc;
  constexpr bool F64 = std::is_same<T, double>::value;
  const Plan& P = h->plan;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  Acc* xt = reinterpret_cast<Acc*>(h->xt.p) + (size_t)kGuard * NR;
  Acc* t = reinterpret_cast<Acc*>(h->tbuf.p) + (size_t)kGuard * NR;
  Acc* yl = reinterpret_cast<Acc*>(h->ylev.p);
  cudaEvent_t ev[5];
  const bool prof = h->profiling;
  if (prof) {
    HD_TRY(chunk_events(h, ev));
    HD_CUDA(cudaEventRecord(ev[0], st));
  }
  const bool packed = !F64 && NR == 1 && ldx == 1 && c0 == 0 && h->d <= 3 && P.rel4_ptrs.n > 0;
  if (packed) {
    if constexpr (NR == 1 && !F64)
      k_gather_pack<IO><<<(int)std::min<int64_t>((h->N + 255) / 256, sms * 16), 256, 0, st>>>(
          x, h->perm.p, h->N, ldx, c0, reinterpret_cast<float*>(xt), P.rel4_ptrs.p, (int)P.rel4_ptrs.n);
  } else {
    k_gather<Acc, IO, NR><<<(int)std::min<int64_t>((h->N + 255) / 256, sms * 16), 256, 0, st>>>(x, h->perm.p, h->N,
                                                                                                ldx, c0, xt);
  }
  h->launches += 1;
  if (prof) HD_CUDA(cudaEventRecord(ev[1], st));
  const size_t smem = (size_t)kStages * kSlotBytes;
  if (h->kappa >= 1) {
    HD_CUDA(cudaMemsetAsync(yl, 0, (size_t)h->kappa * h->N * NR * sizeof(Acc), st));
    if (P.vs.ctas > 0 && !P.vs.h_stages.empty()) {
      k_segdot<T, NR><<<P.vs.ctas, kSegThreads, smem, st>>>(
          reinterpret_cast<const T*>(P.vs.data.p), P.vs.groups.p, P.vs.stages.p, P.vs.cta.p, xt, t,
          Fac<T>::scaled ? h->sv.p : nullptr, Fac<T>::scaled ? h->su.p : nullptr, h->err.p);
      h->launches += 1;
    }
  }
  if (prof) HD_CUDA(cudaEventRecord(ev[2], st));
  if (h->kappa >= 1 && P.us.ctas > 0 && !P.us.h_stages.empty()) {
    k_ucols<T, NR><<<P.us.ctas, kSegThreads, usmem<T, NR>(), st>>>(reinterpret_cast<const T*>(P.us.data.p),
                                                                 P.us.panels.p, P.us.stages.p, P.us.cta.p, t, yl,
                                                                 h->err.p);
    h->launches += 1;
  }
  if (prof) HD_CUDA(cudaEventRecord(ev[3], st));
  if (packed) {
    if constexpr (NR == 1 && !F64) HD_TRY((launch_dense4<IO>(h, st, sms, yl, y, ldx, c0)));
  } else switch (h->d) {
    case 1: HD_TRY((launch_dense<Acc, IO, NR, 1, F64>(h, st, sms, xt, yl, y, ldx, c0))); break;
    case 2: HD_TRY((launch_dense<Acc, IO, NR, 2, F64>(h, st, sms, xt, yl, y, ldx, c0))); break;
    case 3: HD_TRY((launch_dense<Acc, IO, NR, 3, F64>(h, st, sms, xt, yl, y, ldx, c0))); break;
    case 4: HD_TRY((launch_dense<Acc, IO, NR, 4, F64>(h, st, sms, xt, yl, y, ldx, c0))); break;
    default: HD_TRY((launch_dense<Acc, IO, NR, 0, F64>(h, st, sms, xt, yl, y, ldx, c0))); break;
  }
  if (prof) HD_CUDA(cudaEventRecord(ev[4], st));
  HD_CUDA(cudaGetLastError());
  return HODLRDD_OK;
}

template <class T>
int set_smem_attr() {
  static bool done = false;
  if (done) return HODLRDD_OK;
  const int smem = kStages * kSlotBytes;
  HD_CUDA(cudaFuncSetAttribute(k_segdot<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  HD_CUDA(cudaFuncSetAttribute(k_segdot<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  HD_CUDA(cudaFuncSetAttribute(k_segdot<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  HD_CUDA(cudaFuncSetAttribute(k_segdot<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  HD_CUDA(cudaFuncSetAttribute(k_ucols<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)usmem<T, 1>()));
  HD_CUDA(cudaFuncSetAttribute(k_ucols<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)usmem<T, 2>()));
  HD_CUDA(cudaFuncSetAttribute(k_ucols<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)usmem<T, 4>()));
  HD_CUDA(cudaFuncSetAttribute(k_ucols<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)usmem<T, 8>()));
  done = true;
  return HODLRDD_OK;
}

template <class T, class IO>
int matvec_typed(hodlrdd_s* h, const IO* x, IO* y, int nrhs, cudaStream_t st) {
  HD_TRY(set_smem_attr<T>());
  int c0 = 0;
  while (c0 < nrhs) {
    const int rem = nrhs - c0;
    if (rem >= 8) { HD_TRY((matvec_chunk<T, IO, 8>(h, x, y, nrhs, c0, st))); c0 += 8; }
    else if (rem >= 4) { HD_TRY((matvec_chunk<T, IO, 4>(h, x, y, nrhs, c0, st))); c0 += 4; }
    else if (rem >= 2) { HD_TRY((matvec_chunk<T, IO, 2>(h, x, y, nrhs, c0, st))); c0 += 2; }
    else { HD_TRY((matvec_chunk<T, IO, 1>(h, x, y, nrhs, c0, st))); c0 += 1; }
  }
  return HODLRDD_OK;
}

}  // namespace

int launch_matvec(hodlrdd_s* h, const void* x, void* y, int nrhs, cudaStream_t st) {
  switch (h->opt.precision) {
    case HODLRDD_PREC_FP64:
      return matvec_typed<double, double>(h, static_cast<const double*>(x), static_cast<double*>(y), nrhs, st);
    case HODLRDD_PREC_FP32:
      return matvec_typed<float, float>(h, static_cast<const float*>(x), static_cast<float*>(y), nrhs, st);
    case HODLRDD_PREC_FP16:
      return matvec_typed<__half, float>(h, static_cast<const float*>(x), static_cast<float*>(y), nrhs, st);
    default:
      return matvec_typed<__nv_bfloat16, float>(h, static_cast<const float*>(x), static_cast<float*>(y), nrhs, st);
  }
}

namespace {
template <class T>
int unpack_typed(hodlrdd_s* h, int64_t b, double* U, double* V) {
  const int p = h->h_rank[b];
  if (p == 0) return HODLRDD_OK;
  const Plan& P = h->plan;
  const int64_t c0 = h->h_toff[b];
  std::vector<float> su(p, 1.0f), sv(p, 1.0f);
  HD_CUDA(cudaMemcpy(su.data(), h->su.p + c0, p * sizeof(float), cudaMemcpyDeviceToHost));
  HD_CUDA(cudaMemcpy(sv.data(), h->sv.p + c0, p * sizeof(float), cudaMemcpyDeviceToHost));
  const int m = h->h_bm[b], n = h->h_bn[b];
  if (V) {
    const SegGroup& G = P.vs.h_groups[P.h_vgroup[b]];
    const int a = h->h_bJ0[b] - G.vec;  // lead pad
    std::vector<T> buf((size_t)G.L * G.cnt);
    HD_CUDA(cudaMemcpy(buf.data(), reinterpret_cast<const T*>(P.vs.data.p) + G.off, buf.size() * sizeof(T),
                       cudaMemcpyDeviceToHost));
    for (int k = 0; k < p; ++k)
      for (int j = 0; j < n; ++j) V[(size_t)k * n + j] = Fac<T>::to_host(buf[(size_t)k * G.L + a + j]) * sv[k];
  }
  if (U) {
    // the box's panels are consecutive; the block's columns start at h_ucol[b]
    for (int r0 = 0; r0 < m; r0 += kPanelRows) {
      const Panel& Pn = P.us.h_panels[P.h_ugroup[b] + r0 / kPanelRows];
      std::vector<T> buf((size_t)Pn.ld * p);
      HD_CUDA(cudaMemcpy(buf.data(), reinterpret_cast<const T*>(P.us.data.p) + Pn.off + (int64_t)P.h_ucol[b] * Pn.ld,
                         buf.size() * sizeof(T), cudaMemcpyDeviceToHost));
      for (int k = 0; k < p; ++k)
        for (int r = 0; r < Pn.R; ++r)
          U[(size_t)k * m + r0 + r] = Fac<T>::to_host(buf[(size_t)k * Pn.ld + r]) * su[k];
    }
  }
  return HODLRDD_OK;
}
}  // namespace

int unpack_block(hodlrdd_s* h, int64_t b, double* U, double* V) {
  switch (h->opt.precision) {
    case HODLRDD_PREC_FP64: return unpack_typed<double>(h, b, U, V);
    case HODLRDD_PREC_FP32: return unpack_typed<float>(h, b, U, V);
    case HODLRDD_PREC_FP16: return unpack_typed<__half>(h, b, U, V);
    default: return unpack_typed<__nv_bfloat16>(h, b, U, V);
  }
}

int read_error_word(hodlrdd_s* h, int32_t* code) {
  *code = 0;
  if (!h->err.p) return HODLRDD_OK;
  HD_CUDA(cudaDeviceSynchronize());
  HD_CUDA(cudaMemcpy(code, h->err.p, sizeof(int32_t), cudaMemcpyDeviceToHost));
  return HODLRDD_OK;
}

}  // namespace hd
