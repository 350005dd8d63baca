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
// producer lane moves 48 KB stages with cp.async.bulk into a shared-memory ring
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
    case HODLRDD_PREC_FP32:
    case HODLRDD_PREC_FP32_FP16: return 4;  // the FP16 tail is counted separately
    default: return 2;
  }
}

namespace {

constexpr int kStageBytes = 49152;
constexpr int kConsumerWarps = 16;
constexpr int kSegThreads = 32 * (1 + kConsumerWarps);
constexpr int kPanelRows = 512;                // rows per U panel
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
// L2 policy for data read exactly once per matvec (the factor streams): evict
// it first, so the vectors and descriptors the kernels reuse stay resident.
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void bulk_g2s_once(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Stage descriptors reach a producer warp 32 at a time (lane i holds one), one
// batch ahead of use, so no stage waits on a descriptor load.
struct StageRegs {
  int2 w[5];
};
static_assert(sizeof(Stage) == 40, "Stage is five 8-byte words");
__device__ __forceinline__ void load_stage_regs(StageRegs& r, const Stage* __restrict__ s, int q, int q1) {
  if (q < q1) {
    const int2* p = reinterpret_cast<const int2*>(s + q);
#pragma unroll
    for (int k = 0; k < 5; ++k) r.w[k] = __ldg(p + k);
  } else {
#pragma unroll
    for (int k = 0; k < 5; ++k) r.w[k] = make_int2(0, 0);
  }
}
// Stage k (0 <= k < 64) of the batches a (k < 32) and b (k >= 32), to every
// lane; k is warp-uniform.
__device__ __forceinline__ Stage pick_stage(const StageRegs& a, const StageRegs& b, int k) {
  int2 w[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int x = k < 32 ? a.w[i].x : b.w[i].x, y = k < 32 ? a.w[i].y : b.w[i].y;
    w[i] = make_int2(__shfl_sync(0xffffffffu, x, k & 31), __shfl_sync(0xffffffffu, y, k & 31));
  }
  Stage st;
  memcpy(&st, w, sizeof st);
  return st;
}

__device__ __forceinline__ void consumer_bar() {
  asm volatile("bar.sync 1, %0;" ::"n"(32 * kConsumerWarps) : "memory");
}

// ------------------------------------------------------------- panel apply ----
// Both low-rank applies are the same operation on a "panel": a matrix stored
// as P consecutive lines of ld elements (ld a multiple of 16 bytes), and
//   out[w] = sum_k line_k[w] * s_k      for w < R,
// where s_k is the vector value of line k (NR right-hand sides).
//   U-apply: a panel is rows [r0, r0 + R) of one box's U at one level, stored
//            column-major over the concatenated columns of the box's low-rank
//            IL blocks; line k = column k, s_k = t[vfirst + k], outputs are the
//            contiguous ylev rows out0 + w.
//   V-apply: a panel is up to vpanel_width<T>() consecutive columns of the
//            concatenated V factors of all low-rank IL blocks that share one
//            source box J, stored row-major; line k = source point J0 + k,
//            s_k = x_t[vfirst + k], output w is t[map[out0 + w]].
// Threads own fixed 16-byte chunks of a line (rc) and a residue class of lines
// (cg), so no reduction happens until the panel ends. Long panels are cut into
// sub-panels of at most kSplitBytes so that CTAs get balanced work; a cut
// panel writes per-sub-panel partial sums that k_combine adds in order.
//
// Per stage the producer bulk-copies the lines and their vector values into
// the slot (the values with a lead pad to keep the copy 16-byte aligned), so
// the consumers read only shared memory.
constexpr int kMaxLines = 256;      // lines per stage (bounds the staged vector values)
// V panels are one 16-byte chunk per consumer thread wide, so each thread
// owns its columns over all rows and a panel needs no cross-thread reduction.
template <class T>
constexpr int vpanel_width() {
  return kConsumerWarps * 32 * Fac<T>::E;
}
constexpr int kMetaBytes = 128;     // {Stage, Panel, lead pad}
constexpr int kDynSmemMax = 232448 - 1024;

template <class T, int NR>
struct PanelCfg {
  using Acc = typename Fac<T>::acc;
  static constexpr int kScal = kMaxLines * NR * (int)sizeof(Acc) + 16;
  static constexpr int kSlot = kStageBytes + kScal + kMetaBytes;
  static constexpr int kRed = kConsumerWarps * 32 * 8 * (int)sizeof(Acc);
  static constexpr int kFit = (kDynSmemMax - kRed) / kSlot;
  // three slots keep 144 KB in flight per SM and leave shared memory and
  // registers for one near-field tile CTA beside the panel CTA (fewer, larger
  // stages than four of 32 KB: the per-stage hand-over costs the consumers
  // about as many instructions as a 32 KB stage's arithmetic)
  static constexpr int kStagesN = kFit < 3 ? kFit : 3;
  static constexpr size_t kSmem = (size_t)kStagesN * kSlot + kRed;
  static_assert(kStagesN >= 3, "panel ring needs at least three slots");
  // a CTA that reserves the whole SM (the near field on SMs of its own) has
  // room for a fourth slot: 192 KB in flight, for fewer CTAs streaming the
  // same bytes
  static constexpr int kStagesWide = kFit < 4 ? kFit : 4;
  static constexpr size_t smem(int ns) { return (size_t)ns * kSlot + kRed; }
};

// A panel CTA's dynamic shared memory when it reserves a whole SM: the
// per-block limit less 512 bytes for its static shared memory (the mbarriers,
// 128 bytes as compiled); what stays free of the SM's 228 KB is less than the
// 1 KB every CTA reserves, so no other CTA fits beside it
constexpr size_t panel_smem_full() { return (size_t)232448 - 512; }

struct PanelMeta {
  Stage st;
  Panel P;
  int32_t lead;  // elements of lead pad before the first staged vector value
};
static_assert(sizeof(PanelMeta) <= kMetaBytes, "panel metadata exceeds its slot area");

// One stream's arguments (factor data, sub-panels, stages, CTA ranges, vector
// in, outputs, V column map and scales, partial sums).
template <class T>
struct PanelArgs {
  using Acc = typename Fac<T>::acc;
  const T* F;
  const Panel* panels;
  const Stage* stages;
  const int32_t* cta_first;
  int ctas;
  const Acc* vec;
  Acc* out;
  const int32_t* map;
  const float* scl;  // V: per output, the product of its column scales (16-bit streams), else null
  Acc* part;
};

// Producer warp: bulk-copies this CTA's stages of one stream into the ring;
// stage descriptors a batch ahead, panel records one stage ahead (registers)
// and eight ahead (L2). `issued` counts every stage the ring has taken, over
// the streams one launch applies. False when a bounded wait expired (the
// copies already issued have then landed).
template <class T, int NR, int NS>
__device__ __forceinline__ bool panel_produce(const PanelArgs<T>& a, char* smem, uint64_t* full, uint64_t* empty,
                                              int& issued, int32_t* err, uint64_t once) {
  using Acc = typename Fac<T>::acc;
  using C = PanelCfg<T, NR>;
  constexpr int A1 = 16 / (int)sizeof(Acc);  // vector elements per 16 bytes
  {
    const int lane = threadIdx.x & 31;
    const int q0 = blockIdx.x < a.ctas ? a.cta_first[blockIdx.x] : 0;
    const int q1 = blockIdx.x < a.ctas ? a.cta_first[blockIdx.x + 1] : 0;
    const Stage* __restrict__ stages = a.stages;
    const Panel* __restrict__ panels = a.panels;
    bool ok = true;
    StageRegs ca, cb;
    load_stage_regs(ca, stages, q0 + lane, q1);
    load_stage_regs(cb, stages, q0 + 32 + lane, q1);
    Stage st_next = pick_stage(ca, cb, 0);
    Panel P_next{};
    if (q0 < q1) P_next = panels[st_next.g];
    for (int q = q0, j = 0; q < q1; ++q, ++j, ++issued) {
      const int k = j & 31;
      const Stage st = st_next;
      const Panel Pq = P_next;
      if (q + 1 < q1) {
        st_next = pick_stage(ca, cb, k + 1);
        P_next = panels[st_next.g];
      }
      if (q + 8 < q1) {
        const Stage sp = pick_stage(ca, cb, k + 8);
        if (lane == 0) prefetch_l2(panels + sp.g);
      }
      if (k == 31) {
        ca = cb;
        load_stage_regs(cb, stages, q + 33 + lane, q1);
      }
      const int slot = issued % NS;
      const int use = issued / NS;
      if (use > 0) {
        int w = 1;
        if (lane == 0) w = mbar_wait(&empty[slot], (use - 1) & 1, err, ERR_WAIT_EMPTY) ? 1 : 0;
        if (!__shfl_sync(0xffffffffu, w, 0)) {
          ok = false;
          break;
        }
      }
      if (lane == 0) {
        char* base = smem + (size_t)slot * C::kSlot;
        PanelMeta* meta = reinterpret_cast<PanelMeta*>(base + kStageBytes + C::kScal);
        const int64_t v0 = ((int64_t)Pq.vfirst + st.s) * NR;
        const int la = (int)(v0 % A1);
        meta->st = st;
        meta->P = Pq;
        meta->lead = la;
        __threadfence_block();
        const uint32_t fbytes = (uint32_t)st.nelem * sizeof(T);
        const uint32_t sbytes = (uint32_t)(((la + st.nseg * NR) * (int)sizeof(Acc) + 15) & ~15);
        mbar_expect_tx(&full[slot], fbytes + sbytes);
        bulk_g2s_once(base, a.F + st.off, fbytes, &full[slot], once);
        bulk_g2s(base + kStageBytes, a.vec + (v0 - la), sbytes, &full[slot]);
      }
      __syncwarp();
    }
    if (!ok && lane == 0) {
      // drain: copies already issued must land before the CTA's smem goes away
      for (int k = max(0, issued - NS); k < issued; ++k) mbar_wait(&full[k % NS], (k / NS) & 1, err, ERR_WAIT_DRAIN);
    }
    return ok;
  }

}

// Consumer warps: apply this CTA's stages of one stream; ibase = the ring index
// of its first stage. False when a bounded wait expired.
template <class T, int NR, bool VMODE, int NS>
__device__ __forceinline__ bool panel_consume(const PanelArgs<T>& a, char* smem, uint64_t* full, uint64_t* empty,
                                              typename Fac<T>::acc* red, int ibase, int32_t* err) {
  using Acc = typename Fac<T>::acc;
  using C = PanelCfg<T, NR>;
  constexpr int E = Fac<T>::E;
  constexpr int NT = kConsumerWarps * 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q0 = blockIdx.x < a.ctas ? a.cta_first[blockIdx.x] : 0;
  const int q1 = blockIdx.x < a.ctas ? a.cta_first[blockIdx.x + 1] : 0;
  const int32_t* __restrict__ map = a.map;
  const float* __restrict__ scl = a.scl;
  Acc* __restrict__ part = a.part;
  Acc* __restrict__ out = a.out;
  const int cw = warp - 1;
  const int ct = cw * 32 + lane;
  // FP32 with one or two right-hand sides: plain sums over up to kKahanStages
  // stages, added to the total with compensation (Kahan); otherwise plain
  // accumulation (register budget)
  constexpr bool KAHAN = std::is_same<T, float>::value && NR <= 2;
  constexpr int kKahanStages = 4;
  Acc acc[E][NR], cmp[E][NR], sum[E][NR];
  int nsum = 0;
#pragma unroll
  for (int e = 0; e < E; ++e)
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      acc[e][r] = Acc(0);
      cmp[e][r] = Acc(0);
      sum[e][r] = Acc(0);
    }
  // V-apply writers (line class 0) fetch their output indices and scales when
  // a panel starts, so the panel's end does not wait on them
  int32_t oidx[VMODE ? E : 1];
  Acc oscl[VMODE ? E : 1];
  for (int q = q0; q < q1; ++q) {
    const int i = ibase + (q - q0);
    const int slot = i % NS;
    if (!mbar_wait(&full[slot], (i / NS) & 1, err, ERR_WAIT_FULL)) return false;
    const char* base = smem + (size_t)slot * C::kSlot;
    const PanelMeta* meta = reinterpret_cast<const PanelMeta*>(base + kStageBytes + C::kScal);
    const Stage st = meta->st;
    const Panel P = meta->P;
    const Acc* sv = reinterpret_cast<const Acc*>(base + kStageBytes) + meta->lead;
    // chunks per line RC, rounded up to a power of two 2^lg; line classes NT / 2^lg
    const int RC = P.ld / E;
    const int lg = RC > 1 ? 32 - __clz(RC - 1) : 0;
    const int RCP = 1 << lg;
    const int CG = NT >> lg;
    const int rc = ct & (RCP - 1), cg = ct >> lg;
    if (st.ng) {
#pragma unroll
      for (int e = 0; e < E; ++e)
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          acc[e][r] = Acc(0);
          cmp[e][r] = Acc(0);
          sum[e][r] = Acc(0);
        }
      nsum = 0;
      if constexpr (VMODE) {
        if (cg == 0 && rc < RC && P.part < 0) {
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int w = rc * E + e;
            // two independent loads, first used when the panel ends
            oidx[e] = w < P.R ? map[(int64_t)P.out0 + w] : 0;
            oscl[e] = (scl && w < P.R) ? (Acc)scl[(int64_t)P.out0 + w] : Acc(1);
          }
        }
      }
    }
    if (rc < RC) {
      if constexpr (KAHAN) {
#pragma unroll 4
        for (int k = cg; k < st.nseg; k += CG) {
          Acc f[E];
          Fac<T>::chunk(base + ((int64_t)k * P.ld + (int64_t)rc * E) * sizeof(T), f);
#pragma unroll
          for (int e = 0; e < E; ++e)
#pragma unroll
            for (int r = 0; r < NR; ++r) sum[e][r] += f[e] * sv[k * NR + r];
        }
        if (++nsum == kKahanStages || st.last) {
#pragma unroll
          for (int e = 0; e < E; ++e)
#pragma unroll
            for (int r = 0; r < NR; ++r) {
              const Acc y = sum[e][r] - cmp[e][r];
              const Acc s2 = acc[e][r] + y;
              cmp[e][r] = (s2 - acc[e][r]) - y;
              acc[e][r] = s2;
              sum[e][r] = Acc(0);
            }
          nsum = 0;
        }
      } else if constexpr ((NR * sizeof(Acc)) % 16 == 0) {
        // a line's NR vector values are 16-byte aligned (the lead pad is zero
        // when NR values fill whole 16-byte units): vector loads, and one line
        // per iteration so that the NR x E accumulators stay in registers
        constexpr int VW = 16 / (int)sizeof(Acc);
        using Vec = typename std::conditional<sizeof(Acc) == 4, float4, double2>::type;
#pragma unroll 1
        for (int k = cg; k < st.nseg; k += CG) {
          Acc f[E];
          Fac<T>::chunk(base + ((int64_t)k * P.ld + (int64_t)rc * E) * sizeof(T), f);
          const Vec* v4 = reinterpret_cast<const Vec*>(sv + k * NR);
#pragma unroll
          for (int r4 = 0; r4 < NR / VW; ++r4) {
            const Vec vv = v4[r4];
            Acc xv[VW];
            if constexpr (VW == 4) {
              xv[0] = vv.x; xv[1] = vv.y; xv[2] = vv.z; xv[3] = vv.w;
            } else {
              xv[0] = vv.x; xv[1] = vv.y;
            }
#pragma unroll
            for (int e = 0; e < E; ++e)
#pragma unroll
              for (int r = 0; r < VW; ++r) acc[e][r4 * VW + r] += f[e] * xv[r];
          }
        }
      } else {
#pragma unroll 4
        for (int k = cg; k < st.nseg; k += CG) {
          Acc f[E];
          Fac<T>::chunk(base + ((int64_t)k * P.ld + (int64_t)rc * E) * sizeof(T), f);
#pragma unroll
          for (int e = 0; e < E; ++e)
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[e][r] += f[e] * sv[k * NR + r];
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
      // sum the CG line classes: lanes of one warp first, then across warps
      for (int o = 16; o >= RCP; o >>= 1)
#pragma unroll
        for (int e = 0; e < E; ++e)
#pragma unroll
          for (int r = 0; r < NR; ++r) acc[e][r] += __shfl_xor_sync(0xffffffffu, acc[e][r], o);
      const int lw = lg > 5 ? lg - 5 : 0;      // log2 of the warps per line class
      const int WG = 1 << lw;
      const int NG = kConsumerWarps >> lw;     // line classes left after the warp step
      const int sub = cw & (WG - 1), g = cw >> lw;
      const bool holds = lane < (RCP < 32 ? RCP : 32);
      if (NG > 1) {
#pragma unroll
        for (int c0 = 0; c0 < E * NR; c0 += 8) {
          if (holds)
#pragma unroll
            for (int c = 0; c < 8; ++c)
              if (c0 + c < E * NR) red[(int64_t)ct * 8 + c] = acc[(c0 + c) / NR][(c0 + c) % NR];
          consumer_bar();
          if (g == 0 && holds) {
            for (int gg = 1; gg < NG; ++gg)
#pragma unroll
              for (int c = 0; c < 8; ++c)
                if (c0 + c < E * NR)
                  acc[(c0 + c) / NR][(c0 + c) % NR] += red[(int64_t)((gg * WG + sub) * 32 + lane) * 8 + c];
          }
          consumer_bar();
        }
      }
      const int orc = sub * 32 + lane;  // chunk held after the reduction
      if (g == 0 && holds && orc < RC) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int w = orc * E + e;
          if (w < P.R) {
            if (P.part >= 0) {
#pragma unroll
              for (int r = 0; r < NR; ++r) part[((int64_t)P.part + w) * NR + r] = acc[e][r];
            } else if constexpr (VMODE) {
#pragma unroll
              for (int r = 0; r < NR; ++r) out[(int64_t)oidx[e] * NR + r] = acc[e][r] * oscl[e];
            } else {
#pragma unroll
              for (int r = 0; r < NR; ++r) out[((int64_t)P.out0 + w) * NR + r] = acc[e][r];
            }
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[slot]);
  }
  return true;
}

template <int NR>
__device__ __forceinline__ void panel_ring_init(uint64_t* full, uint64_t* empty, int ns) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}

// NS: ring slots (PanelCfg::kStagesN, or kStagesWide when the CTA holds a whole SM)
template <class T, int NR, bool VMODE, int NS>
__global__ void __launch_bounds__(kSegThreads, 1) k_panel(PanelArgs<T> a, int32_t* __restrict__ err) {
  using C = PanelCfg<T, NR>;
  extern __shared__ __align__(128) char smem[];
  __shared__ __align__(8) uint64_t full[NS], empty[NS];
  auto* red = reinterpret_cast<typename Fac<T>::acc*>(smem + (size_t)NS * C::kSlot);  // NT * 8
  panel_ring_init<NR>(full, empty, NS);
  if ((threadIdx.x >> 5) == 0) {
    int issued = 0;
    panel_produce<T, NR, NS>(a, smem, full, empty, issued, err, l2_evict_first());
    return;
  }
  panel_consume<T, NR, VMODE, NS>(a, smem, full, empty, red, 0, err);
}

// Mixed storage: one launch applies the FP32 stream and then the FP16 stream of
// the same stage through one ring (both have the same slot layout), so that the
// two parts share one persistent CTA per SM instead of following each other.
template <int NR, bool VMODE, int NS>
__global__ void __launch_bounds__(kSegThreads, 1) k_panel_mix(PanelArgs<float> a, PanelArgs<__half> b,
                                                              int32_t* __restrict__ err) {
  using C = PanelCfg<float, NR>;
  static_assert(C::kSlot == PanelCfg<__half, NR>::kSlot && C::kStagesN == PanelCfg<__half, NR>::kStagesN &&
                    C::kStagesWide == PanelCfg<__half, NR>::kStagesWide,
                "the two element types must share the ring layout");
  extern __shared__ __align__(128) char smem[];
  __shared__ __align__(8) uint64_t full[NS], empty[NS];
  float* red = reinterpret_cast<float*>(smem + (size_t)NS * C::kSlot);
  panel_ring_init<NR>(full, empty, NS);
  if ((threadIdx.x >> 5) == 0) {
    const uint64_t once = l2_evict_first();
    int issued = 0;
    if (!panel_produce<float, NR, NS>(a, smem, full, empty, issued, err, once)) return;
    panel_produce<__half, NR, NS>(b, smem, full, empty, issued, err, once);
    return;
  }
  const int na = blockIdx.x < a.ctas ? a.cta_first[blockIdx.x + 1] - a.cta_first[blockIdx.x] : 0;
  if (!panel_consume<float, NR, VMODE, NS>(a, smem, full, empty, red, 0, err)) return;
  panel_consume<__half, NR, VMODE, NS>(b, smem, full, empty, red, na, err);
}

// Sums of cut panels: out = sum over the sub-panels' partials, in sub-panel
// order; V outputs go through the column map and the column scales. One CTA
// per (split, block of kCombineRows outputs) work item.
constexpr int kCombineRows = 256;

template <class Acc, int NR, bool VMODE>
__global__ void __launch_bounds__(256) k_combine(const Split* __restrict__ splits, const int2* __restrict__ work,
                                                  const Acc* __restrict__ part, Acc* __restrict__ out,
                                                  const int32_t* __restrict__ map, const float* __restrict__ sa,
                                                  const float* __restrict__ sb) {
  const int2 wk = work[blockIdx.x];
  const Split S = splits[wk.x];
  const int w1 = min(S.R, wk.y + kCombineRows);
  for (int idx = threadIdx.x; idx < (w1 - wk.y) * NR; idx += blockDim.x) {
    const int w = wk.y + idx / NR, r = idx % NR;
    Acc v = Acc(0);
    for (int s = 0; s < S.nsplit; ++s) v += part[((int64_t)S.part + (int64_t)s * S.R + w) * NR + r];
    if constexpr (VMODE) {
      const int64_t o = map[(int64_t)S.out0 + w];
      const Acc sc = sa ? (Acc)(sa[o] * sb[o]) : Acc(1);
      out[o * NR + r] = v * sc;
    } else {
      out[((int64_t)S.out0 + w) * NR + r] = v;
    }
  }
}

// ------------------------------------------------------------- dense ----
// One CTA (256 threads) per task (target rows [I0, I0+m) at one level). Rows
// are handled G at a time (G a power of two up to 256) with 256 / G source
// stripes; each stripe's partial sums meet in shared memory and are added in
// stripe order (fixed, so products are bitwise reproducible). A CTA, not a
// warp, per task: small trees (C1: 256 leaf tasks) would otherwise leave most
// SMs idle while each warp walks its task's sources alone. Box-relative FP32
// coordinates: x_i - x_j = (rel_i - rel_j) + (c_I - c_J) h, where the box
// offset is exact in FP32, so differences keep full FP32 accuracy at the box
// scale. The FP64 form uses the global FP64 coordinates.
template <class Acc, class IO, int NR, int D, bool F64, bool FINAL>
__global__ void __launch_bounds__(256) k_dense(const int4* __restrict__ tasks, int64_t t0, int64_t t1,
                                               const int2* __restrict__ srcs, const float* __restrict__ soff,
                                               const float* __restrict__ rel, const double* __restrict__ p64,
                                               int64_t N, int d_rt, int kid, double kc, double kscale, double kdiag,
                                               const Acc* __restrict__ xt, Acc* __restrict__ ylev_l,
                                               const Acc* __restrict__ ylev, int kappa,
                                               const int32_t* __restrict__ perm, IO* __restrict__ y, int ldy,
                                               int c0) {
  constexpr int NT = 256;
  __shared__ Acc red[NT * NR];
  const int d = D > 0 ? D : d_rt;
  const int tid = threadIdx.x;
  const float kcf = (float)kc;
  for (int64_t it = t0 + blockIdx.x; it < t1; it += gridDim.x) {
    const int4 task = tasks[it];
    const int I0 = task.x, m = task.y;
    int G = 1;
    while (G < m && G < NT) G <<= 1;
    const int S = NT / G;
    const int gi = tid % G, stripe = tid / G;
    for (int g0 = 0; g0 < m; g0 += G) {
      const int row = I0 + g0 + gi;
      const bool valid = g0 + gi < m;
      Acc acc[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[r] = Acc(0);
      if (valid) {
        if constexpr (F64) {
          double xr[D > 0 ? D : kMaxDim];
          for (int k = 0; k < d; ++k) xr[k] = p64[(int64_t)k * N + row];
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
          for (int k = 0; k < d; ++k) xr[k] = rel[(int64_t)k * N + row];
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
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) red[tid * NR + r] = acc[r];
      __syncthreads();
      if (stripe == 0 && valid) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          Acc a = Acc(0);
          for (int q = 0; q < S; ++q) a += red[(q * G + gi) * NR + r];
          acc[r] = a;
        }
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
      __syncthreads();  // red is reused by the next rows
    }
  }
}

// Packed near field / dense blocks (FP32, d <= 3, one right-hand side): a
// point is one float4 (box-relative coordinates, x_t in .w); a source box is an
// int4 {J0, n} and its exact box offset; the kernel function is a template
// parameter so the pair loop has no branch on it.
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
// Column source offsets in the FP64 ACA output: colU[c] / colV[c] for the t
// index c of ACA column k of block b: c = thead[b] + k for k < kb[b] (the
// leading columns), ttail[b] + k - kb[b] for the others.
__global__ void k_colmap(int64_t nblk, const int32_t* __restrict__ rank, const int32_t* __restrict__ bm,
                         const int32_t* __restrict__ bn, const int32_t* __restrict__ kb,
                         const int64_t* __restrict__ thead, const int64_t* __restrict__ ttail,
                         const int64_t* __restrict__ uoff64, const int64_t* __restrict__ voff64,
                         int64_t* __restrict__ colU, int64_t* __restrict__ colV) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < rank[b]; ++k) {
      const int64_t c = k < kb[b] ? thead[b] + k : ttail[b] + (k - kb[b]);
      colU[c] = uoff64[b] + (int64_t)k * bm[b];
      colV[c] = voff64[b] + (int64_t)k * bn[b];
    }
}

// ||u_c||_2 ||v_c||_2 per column (one warp per column).
__global__ void k_termnorm(int64_t ncol, const int64_t* __restrict__ colU, const int64_t* __restrict__ colV,
                           const int32_t* __restrict__ colrows_u, const int32_t* __restrict__ colrows_v,
                           const double* __restrict__ U64, const double* __restrict__ V64, double* __restrict__ tn) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = warp; c < ncol; c += nw) {
    double su = 0.0, sv = 0.0;
    for (int i = lane; i < colrows_u[c]; i += 32) su = fma(U64[colU[c] + i], U64[colU[c] + i], su);
    for (int i = lane; i < colrows_v[c]; i += 32) sv = fma(V64[colV[c] + i], V64[colV[c] + i], sv);
    for (int o = 16; o; o >>= 1) {
      su += __shfl_xor_sync(0xffffffffu, su, o);
      sv += __shfl_xor_sync(0xffffffffu, sv, o);
    }
    if (lane == 0) tn[c] = sqrt(su) * sqrt(sv);
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

// U panels: one CTA per whole panel; element (k, w) is row r0 + w of global
// column c0 + k, divided by the column's scale (zero for w >= R).
template <class T>
__global__ void k_packU(int64_t npan, const LPanel* __restrict__ lp, const int32_t* __restrict__ prow0,
                        const int32_t* __restrict__ pcol0, const int64_t* __restrict__ colU,
                        const double* __restrict__ U64, const float* __restrict__ su, T* __restrict__ out) {
  for (int64_t p = blockIdx.x; p < npan; p += gridDim.x) {
    const LPanel L = lp[p];
    const int r0 = prow0[p], c0 = pcol0[p];
    for (int64_t idx = threadIdx.x; idx < (int64_t)L.lines * L.ld; idx += blockDim.x) {
      const int k = (int)(idx / L.ld), w = (int)(idx % L.ld);
      const int64_t c = (int64_t)c0 + k;
      const double v = w < L.R ? U64[colU[c] + r0 + w] / (double)su[c] : 0.0;
      out[L.off + idx] = Fac<T>::from(v);
    }
  }
}

// V panels: one CTA per whole panel; element (k, w) is row k of global column
// map[m0 + w], divided by its scale. 32 x 32 tiles through shared memory keep
// both the column reads and the row writes contiguous.
template <class T>
__global__ void __launch_bounds__(256) k_packV(int64_t npan, const LPanel* __restrict__ lp,
                                               const int32_t* __restrict__ pm0, const int32_t* __restrict__ map,
                                               const int64_t* __restrict__ colV, const double* __restrict__ V64,
                                               const float* __restrict__ sv, T* __restrict__ out) {
  __shared__ double tile[32][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t p = blockIdx.x; p < npan; p += gridDim.x) {
    const LPanel L = lp[p];
    const int m0 = pm0[p];
    for (int k0 = 0; k0 < L.lines; k0 += 32)
      for (int w0 = 0; w0 < L.ld; w0 += 32) {
        for (int ww = warp; ww < 32; ww += 8) {
          const int w = w0 + ww, k = k0 + lane;
          double v = 0.0;
          if (w < L.R && k < L.lines) {
            const int64_t c = map[m0 + w];
            v = V64[colV[c] + k] / (double)sv[c];
          }
          tile[ww][lane] = v;
        }
        __syncthreads();
        for (int kk = warp; kk < 32; kk += 8) {
          const int k = k0 + kk, w = w0 + lane;
          if (k < L.lines && w < L.ld) out[L.off + (int64_t)k * L.ld + w] = Fac<T>::from(tile[lane][kk]);
        }
        __syncthreads();
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

// Sub-panels, partial-sum splits and stages of a stream whose whole panels
// (h_lp, with per-panel vector and output origins) are set. A panel longer than
// kSplitBytes is cut into nearly equal sub-panels whose sums k_combine adds; a
// stage holds up to kMaxLines whole lines and at most kStageBytes. CTA ranges
// are balanced by bytes and cut only between sub-panels.
constexpr int64_t kSplitBytes = 1 << 20;

// SMs the persistent apply kernels are scheduled on: all of them, or all but
// near_sms when the single-right-hand-side FP32 near field has SMs of its own
int apply_sms(const hodlrdd_s* h, int sms) {
  const int pr = h->opt.precision;
  const bool own = h->opt.near_sms > 0 && h->opt.lowrank_form == 0 && h->d <= 3 && pr != HODLRDD_PREC_FP64 &&
                   pr != HODLRDD_PREC_FP16X2;
  return own ? std::max(1, sms - h->opt.near_sms) : sms;
}

void balance_ctas(Stream& S, size_t esize, int ctas);

void schedule_stream(Stream& S, const std::vector<int32_t>& vfirst, const std::vector<int32_t>& out0,
                     size_t esize, int ctas) {
  S.h_panels.clear();
  S.h_stages.clear();
  S.h_splits.clear();
  S.part_rows = 0;
  for (size_t p = 0; p < S.h_lp.size(); ++p) {
    const LPanel& L = S.h_lp[p];
    const int64_t line_bytes = (int64_t)L.ld * (int64_t)esize;
    const int64_t maxl = std::max<int64_t>(1, kSplitBytes / line_bytes);
    const int nsplit = (int)std::max<int64_t>(1, (L.lines + maxl - 1) / maxl);
    const int per_split = (L.lines + nsplit - 1) / nsplit;
    int32_t pbase = -1;
    if (nsplit > 1) {
      pbase = (int32_t)S.part_rows;
      S.h_splits.push_back(Split{pbase, nsplit, L.R, out0[p]});
      S.part_rows += (int64_t)nsplit * L.R;
    }
    const int per_stage = (int)std::min<int64_t>(kMaxLines, std::max<int64_t>(1, kStageBytes / line_bytes));
    for (int s = 0, k0 = 0; k0 < L.lines; ++s, k0 += per_split) {
      const int k1 = std::min(L.lines, k0 + per_split);
      const int g = (int)S.h_panels.size();
      S.h_panels.push_back(Panel{L.off + (int64_t)k0 * L.ld, L.ld, L.R, k1 - k0, vfirst[p] + k0, out0[p],
                                 nsplit > 1 ? pbase + s * L.R : -1});
      for (int k = 0; k < k1 - k0; k += per_stage) {
        const int n = std::min(per_stage, k1 - k0 - k);
        S.h_stages.push_back(Stage{L.off + (int64_t)(k0 + k) * L.ld, n * L.ld, g, k, n, -1,
                                   k + n >= k1 - k0 ? 1 : 0, k == 0 ? 1 : 0, 0});
      }
    }
  }
  S.h_cwork.clear();
  for (size_t i = 0; i < S.h_splits.size(); ++i)
    for (int w0 = 0; w0 < S.h_splits[i].R; w0 += kCombineRows) S.h_cwork.push_back(make_int2((int)i, w0));
  balance_ctas(S, esize, ctas);
}

// CTA ranges of a stream's stages, balanced by time, not bytes: a stage costs
// its bytes plus a fixed hand-over (the ring round trip, the end-of-panel
// reduction and the output indices a one-stage panel waits for), about what
// 32 KB take to stream; trees whose finest boxes hold a few points have
// thousands of one-stage panels, and a bytes-only split gave some CTAs twenty
// times the others' time. Ranges end only where a sub-panel ends.
void balance_ctas(Stream& S, size_t esize, int ctas) {
  const int64_t stage_cost = std::max<int64_t>(1, 32768 / esize);
  int64_t total = 0;
  for (const Stage& st : S.h_stages) total += st.nelem + stage_cost;
  S.h_cta.assign(1, 0);
  int64_t acc = 0;
  const int64_t target = std::max<int64_t>(1, (total + ctas - 1) / ctas);
  for (size_t q = 0; q < S.h_stages.size(); ++q) {
    acc += S.h_stages[q].nelem + stage_cost;
    if (S.h_stages[q].last && acc >= target * (int64_t)S.h_cta.size() && (int)S.h_cta.size() < ctas)
      S.h_cta.push_back((int32_t)(q + 1));
  }
  if (S.h_cta.back() != (int32_t)S.h_stages.size()) S.h_cta.push_back((int32_t)S.h_stages.size());
  S.ctas = (int)S.h_cta.size() - 1;
}

int upload_stream(Stream& S, cudaStream_t st) {
  HD_TRY(upload(S.panels, S.h_panels, st));
  HD_TRY(upload(S.stages, S.h_stages, st));
  HD_TRY(upload(S.cta, S.h_cta, st));
  HD_TRY(upload(S.splits, S.h_splits, st));
  HD_TRY(upload(S.cwork, S.h_cwork, st));
  return HODLRDD_OK;
}

// The columns one storage part holds: block b contributes its ACA columns
// [k0[b], k1[b]) with t indices tfirst[b] + (k - k0[b]); the t indices of one
// target box's columns are consecutive (the U-apply reads them as one range).
struct ColPart {
  std::vector<int32_t> k0, k1;
  std::vector<int64_t> tfirst;
};

// Panels of one part in element type T: V per (level, source box), U per
// (level, target box); packs them from the FP64 ACA output. U outputs go to
// y_l slice offset yoff. `track` records the per-block panel positions that
// hodlrdd_get_factors reads back.
template <class T>
int pack_part(hodlrdd_s* h, const DevBuf<double>& U64, const DevBuf<double>& V64, const DevBuf<int64_t>& colU,
              const DevBuf<int64_t>& colV, const ColPart& cp, Stream& vs, Stream& us, DevBuf<int32_t>& vmap,
              bool track, int64_t yoff) {
  cudaStream_t st = h->st;
  constexpr int E = Fac<T>::E;
  const int64_t nblk = h->nblk;
  Plan& P = h->plan;
  auto roundE = [&](int64_t v) { return (v + E - 1) / E * E; };
  auto ncols = [&](int64_t b) { return cp.k1[b] - cp.k0[b]; };
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);

  // V panels: per level and source box, the concatenated columns of its
  // low-rank IL blocks (in block order) in row-major panels of at most
  // vpanel_width<T>() columns; line k = source point J0 + k
  vs.h_lp.clear();
  if (track) {
    P.h_vpanel.assign(nblk, -1);
    P.h_vcol.assign(nblk, 0);
  }
  std::vector<int32_t> hmap, vfirst_v, out0_v;
  int64_t off = 0;
  for (int l = 1; l <= h->kappa; ++l) {
    std::vector<int64_t> bs;
    for (int64_t b = h->h_blk_off[l]; b < h->h_blk_off[l + 1]; ++b)
      if (ncols(b) > 0) bs.push_back(b);
    std::stable_sort(bs.begin(), bs.end(), [&](int64_t a, int64_t b) { return h->h_bJ0[a] < h->h_bJ0[b]; });
    for (size_t i = 0; i < bs.size();) {
      size_t j = i;
      const int32_t J0 = h->h_bJ0[bs[i]], n = h->h_bn[bs[i]];
      const int64_t first = (int64_t)vs.h_lp.size(), m0 = (int64_t)hmap.size();
      for (; j < bs.size() && h->h_bJ0[bs[j]] == J0; ++j) {
        const int64_t b = bs[j];
        if (track) {
          P.h_vpanel[b] = first;
          P.h_vcol[b] = (int32_t)((int64_t)hmap.size() - m0);
        }
        for (int k = 0; k < ncols(b); ++k) hmap.push_back((int32_t)(cp.tfirst[b] + k));
      }
      const int64_t Q = (int64_t)hmap.size() - m0;
      for (int64_t c0 = 0; c0 < Q; c0 += vpanel_width<T>()) {
        const int32_t R = (int32_t)std::min<int64_t>(vpanel_width<T>(), Q - c0);
        const int32_t ld = (int32_t)roundE(R);
        vs.h_lp.push_back(LPanel{off, ld, R, n});
        vfirst_v.push_back(J0);
        out0_v.push_back((int32_t)(m0 + c0));
        off += (int64_t)ld * n;
      }
      i = j;
    }
  }
  vs.elems = off;
  // U panels: per (level, box) with low-rank blocks, rows in panels of at most
  // kPanelRows, column-major over the box's concatenated IL columns
  us.h_lp.clear();
  if (track) {
    P.h_ugroup.assign(nblk, -1);
    P.h_ucol.assign(nblk, 0);
  }
  std::vector<int32_t> prow0, vfirst_u, out0_u;
  off = 0;
  for (int l = 1; l <= h->kappa; ++l) {
    const Level& L = h->lv[l];
    for (int64_t i = 0; i < L.nb; ++i) {
      const int64_t b0 = h->h_blk_off[l] + L.h_iloff[i], b1 = h->h_blk_off[l] + L.h_iloff[i + 1];
      int64_t Pi = 0, tf = -1;
      for (int64_t b = b0; b < b1; ++b)
        if (ncols(b) > 0) {
          if (tf < 0) tf = cp.tfirst[b];
          if (track) {
            P.h_ugroup[b] = (int64_t)us.h_lp.size();
            P.h_ucol[b] = (int32_t)Pi;
          }
          Pi += ncols(b);
        }
      if (Pi == 0) continue;
      const int32_t I0 = L.h_bstart[i], m = L.h_bstart[i + 1] - I0;
      for (int32_t r0 = 0; r0 < m; r0 += kPanelRows) {
        const int32_t R = std::min(kPanelRows, m - r0);
        const int32_t ld = (int32_t)roundE(R);
        us.h_lp.push_back(LPanel{off, ld, R, (int32_t)Pi});
        prow0.push_back(r0);
        vfirst_u.push_back((int32_t)tf);
        out0_u.push_back((int32_t)(yoff + (int64_t)(l - 1) * h->N + I0 + r0));
        off += (int64_t)ld * Pi;
      }
    }
  }
  us.elems = off;
  schedule_stream(vs, vfirst_v, out0_v, sizeof(T), apply_sms(h, sms));
  schedule_stream(us, vfirst_u, out0_u, sizeof(T), apply_sms(h, sms));

  DevBuf<int32_t> dprow0, dpcol0, dvm0;
  DevBuf<LPanel> dvlp, dulp;
  HD_TRY(upload(dprow0, prow0, st));
  HD_TRY(upload(dpcol0, vfirst_u, st));
  HD_TRY(upload(dvm0, out0_v, st));
  HD_TRY(upload(dvlp, vs.h_lp, st));
  HD_TRY(upload(dulp, us.h_lp, st));
  HD_TRY(upload(vmap, hmap, st));
  HD_TRY(vs.data.alloc((size_t)std::max<int64_t>(vs.elems, E) * sizeof(T)));
  HD_TRY(us.data.alloc((size_t)std::max<int64_t>(us.elems, E) * sizeof(T)));
  HD_TRY(upload_stream(vs, st));
  HD_TRY(upload_stream(us, st));
  const int64_t nvp = (int64_t)vs.h_lp.size(), nup = (int64_t)us.h_lp.size();
  if (nvp)
    k_packV<T><<<(int)std::min<int64_t>(nvp, sms * 16), 256, 0, st>>>(
        nvp, dvlp.p, dvm0.p, vmap.p, colV.p, V64.p, h->sv.p, reinterpret_cast<T*>(vs.data.p));
  if (nup)
    k_packU<T><<<(int)std::min<int64_t>(nup, sms * 16), 256, 0, st>>>(
        nup, dulp.p, dprow0.p, dpcol0.p, colU.p, U64.p, h->su.p, reinterpret_cast<T*>(us.data.p));
  HD_CUDA(cudaGetLastError());
  HD_CUDA(cudaStreamSynchronize(st));
  return HODLRDD_OK;
}

// Relative size below which an ACA term is stored in FP16 by the mixed form:
// ||u_k|| ||v_k|| <= 2^-13 ||A_b||_F (estimate), so that the FP16 rounding
// (2^-11 of each entry, power-of-two column scales) of such a term stays below
// 2^-24 of the block, the FP32 rounding of the leading terms.
constexpr double kTailEta = 1.0 / 8192.0;

// Packs the factors: uniform element type T, or (mixed) the leading terms of
// each block in FP32 and its trailing terms (every term after the last one
// above kTailEta of the block) in FP16 with per-column scales.
// scl[c] = sv[map[c]] * su[map[c]]: the product of the column scales of each
// V panel output of a 16-bit stream, so that a panel's writers load it
// directly instead of through the column index.
__global__ void k_vscl(int64_t n, const int32_t* __restrict__ map, const float* __restrict__ sv,
                       const float* __restrict__ su, float* __restrict__ scl) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
    scl[c] = sv[map[c]] * su[map[c]];
}

int fill_vscl(hodlrdd_s* h, const DevBuf<int32_t>& map, DevBuf<float>& scl) {
  HD_TRY(scl.alloc(std::max<size_t>(map.n, 1)));
  if (map.n > 0) {
    k_vscl<<<(int)std::min<int64_t>(((int64_t)map.n + 255) / 256, 4096), 256, 0, h->st>>>((int64_t)map.n, map.p,
                                                                                         h->sv.p, h->su.p, scl.p);
    HD_CUDA(cudaGetLastError());
  }
  return HODLRDD_OK;
}

template <class T>
int pack_typed(hodlrdd_s* h, const DevBuf<double>& U64, const DevBuf<double>& V64,
               const std::vector<int64_t>& uoff64, const std::vector<int64_t>& voff64, bool mixed) {
  cudaStream_t st = h->st;
  const int64_t nblk = h->nblk;
  Plan& P = h->plan;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  if ((int64_t)h->total_rank + 2 * kGuard >= INT32_MAX || 2 * (int64_t)h->kappa * h->N >= INT32_MAX) {
    set_error("problem too large for 32-bit vector indices");
    return HODLRDD_ERR_UNSUPPORTED;
  }
  const int64_t ncol = h->total_rank;
  DevBuf<int64_t> colU, colV, du64, dv64, dthead, dttail;
  DevBuf<int32_t> crows_u, crows_v, dkb;
  HD_TRY(colU.alloc(std::max<int64_t>(ncol, 1)));
  HD_TRY(colV.alloc(std::max<int64_t>(ncol, 1)));
  HD_TRY(upload(du64, uoff64, st));
  HD_TRY(upload(dv64, voff64, st));
  HD_TRY(h->su.alloc(std::max<int64_t>(ncol, 1)));
  HD_TRY(h->sv.alloc(std::max<int64_t>(ncol, 1)));
  // per-block split: leading kb[b] columns (head), the rest (tail)
  std::vector<int32_t> kb(h->h_rank.begin(), h->h_rank.end());
  auto number = [&](std::vector<int64_t>& thead, std::vector<int64_t>& ttail) -> int64_t {
    thead.assign(nblk, 0);
    ttail.assign(nblk, 0);
    int64_t H = 0;
    for (int64_t b = 0; b < nblk; ++b) {
      thead[b] = H;
      H += kb[b];
    }
    int64_t t = H;
    for (int64_t b = 0; b < nblk; ++b) {
      ttail[b] = t;
      t += h->h_rank[b] - kb[b];
    }
    return H;
  };
  auto colmap = [&](const std::vector<int64_t>& thead, const std::vector<int64_t>& ttail) -> int {
    std::vector<int32_t> hcru(std::max<int64_t>(ncol, 1)), hcrv(std::max<int64_t>(ncol, 1));
    for (int64_t b = 0; b < nblk; ++b)
      for (int k = 0; k < h->h_rank[b]; ++k) {
        const int64_t c = k < kb[b] ? thead[b] + k : ttail[b] + (k - kb[b]);
        hcru[c] = h->h_bm[b];
        hcrv[c] = h->h_bn[b];
      }
    HD_TRY(upload(crows_u, hcru, st));
    HD_TRY(upload(crows_v, hcrv, st));
    HD_TRY(upload(dkb, kb, st));
    HD_TRY(upload(dthead, thead, st));
    HD_TRY(upload(dttail, ttail, st));
    if (ncol > 0)
      k_colmap<<<(int)std::min<int64_t>((nblk + 255) / 256, 4096), 256, 0, st>>>(
          nblk, h->rank.p, h->bm.p, h->bn.p, dkb.p, dthead.p, dttail.p, du64.p, dv64.p, colU.p, colV.p);
    HD_CUDA(cudaGetLastError());
    return HODLRDD_OK;
  };
  std::vector<int64_t> thead, ttail;
  int64_t H = number(thead, ttail);
  HD_TRY(colmap(thead, ttail));
  if (mixed && ncol > 0) {
    DevBuf<double> tn;
    HD_TRY(tn.alloc(ncol));
    k_termnorm<<<grid_warps(ncol, sms), 256, 0, st>>>(ncol, colU.p, colV.p, crows_u.p, crows_v.p, U64.p, V64.p, tn.p);
    HD_CUDA(cudaGetLastError());
    std::vector<double> htn;
    HD_TRY(download(htn, tn.p, (size_t)ncol, st));
    HD_CUDA(cudaStreamSynchronize(st));
    for (int64_t b = 0; b < nblk; ++b) {
      const int p = h->h_rank[b];
      double S = 0.0;
      for (int k = 0; k < p; ++k) S += htn[thead[b] + k] * htn[thead[b] + k];
      S = std::sqrt(S);
      int k = p;
      while (k > 0 && htn[thead[b] + k - 1] <= kTailEta * S) --k;
      kb[b] = k;
    }
    H = number(thead, ttail);
    HD_TRY(colmap(thead, ttail));
  }
  P.tail_cols = ncol - H;
  // scales: 1 for FP32 / FP64 columns, a power of two >= the column's largest
  // entry for 16-bit columns
  if (H > 0)
    k_colscale<<<grid_warps(H, sms), 256, 0, st>>>(H, colU.p, colV.p, crows_u.p, crows_v.p, U64.p, V64.p,
                                                   Fac<T>::scaled ? 1 : 0, h->su.p, h->sv.p);
  if (ncol > H)
    k_colscale<<<grid_warps(ncol - H, sms), 256, 0, st>>>(ncol - H, colU.p + H, colV.p + H, crows_u.p + H,
                                                          crows_v.p + H, U64.p, V64.p, 1, h->su.p + H, h->sv.p + H);
  HD_CUDA(cudaGetLastError());
  ColPart head, tail;
  head.k0.assign(nblk, 0);
  head.k1 = kb;
  head.tfirst = thead;
  HD_TRY(pack_part<T>(h, U64, V64, colU, colV, head, P.vs, P.us, P.vmap, !mixed, 0));
  h->factor_bytes = (P.vs.elems + P.us.elems) * (int64_t)sizeof(T) + (Fac<T>::scaled ? 2 * H * 4 : 0);
  P.vscl.release();
  P.vscl2.release();
  if (Fac<T>::scaled) HD_TRY(fill_vscl(h, P.vmap, P.vscl));
  P.vs2 = Stream();
  P.us2 = Stream();
  P.vmap2.release();
  if (mixed) {
    tail.k0 = kb;
    tail.k1.assign(h->h_rank.begin(), h->h_rank.end());
    tail.tfirst = ttail;
    HD_TRY(pack_part<__half>(h, U64, V64, colU, colV, tail, P.vs2, P.us2, P.vmap2, false,
                             (int64_t)h->kappa * h->N));
    HD_TRY(fill_vscl(h, P.vmap2, P.vscl2));
    h->factor_bytes += (P.vs2.elems + P.us2.elems) * 2 + 2 * (ncol - H) * 4;
  }
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
    case HODLRDD_PREC_FP64: return pack_typed<double>(h, U64, V64, uoff64, voff64, false);
    case HODLRDD_PREC_FP32: return pack_typed<float>(h, U64, V64, uoff64, voff64, false);
    case HODLRDD_PREC_FP32_FP16: return pack_typed<float>(h, U64, V64, uoff64, voff64, true);
    case HODLRDD_PREC_FP16: return pack_typed<__half>(h, U64, V64, uoff64, voff64, false);
    case HODLRDD_PREC_FP16X2: return pack_tc(h, U64, V64, uoff64, voff64);
    default: return pack_typed<__nv_bfloat16>(h, U64, V64, uoff64, voff64, false);
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
  // Packed plan (FP32 arithmetic, d <= 3, one right-hand side): one CTA per
  // task of at most kTileRows rows; sources staged in chunks of kTileCap points.
  std::vector<int4> t4, s4;
  std::vector<float4> o4;                  // per source entry: (c_J - c_I) h_l
  std::vector<char> need4(h->kappa + 1, 0);
  if (h->opt.lowrank_form == 1)  // the FP32 skeleton form evaluates every level's low-rank blocks
    for (int l = 1; l <= h->kappa; ++l) need4[l] = 1;
  std::vector<std::pair<int2, float4>> sl; // current task's sources: {J0, n}, offset
  P.packed_pairs = 0;
  // rows per task: kTileRows, halved (down to 64) while the leaf pass would
  // have fewer than eight tasks per SM, so that trees with few large parent
  // boxes (high d, large leaves) still spread over every SM
  int32_t rows_cap = kTileRows;
  // the tensor-core near field takes tiles of 128 target rows (the MMA's M)
  const bool tc_tiles = h->opt.precision == HODLRDD_PREC_FP16X2 && tc_near_kernel(h->K.id);
  if (tc_tiles) rows_cap = 128;
  if (h->kappa >= 1 && !tc_tiles) {
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    const Level& LP = h->lv[h->kappa - 1];
    auto leaf_tasks = [&](int32_t rows) {
      int64_t n = 0;
      for (int64_t pb = 0; pb < LP.nb; ++pb) n += (LP.h_bstart[pb + 1] - LP.h_bstart[pb] + rows - 1) / rows;
      return n;
    };
    while (rows_cap > 64 && leaf_tasks(rows_cap) < 8 * (int64_t)sms) rows_cap /= 2;
  }
  // tensor-core tiles: each task's target box, and after packing per task its
  // box records and per source entry the boxes of its task that read it
  std::vector<int64_t> tbox_of;  // parallel to t4 (before packing)
  std::vector<int2> tb4;         // parallel to t4 (after packing): {first record, records}
  std::vector<int32_t> brow4;    // record: first row of the box within its task
  std::vector<float4> boff4;     // record: (c_box - c_frame) h_l, the box's offset in the task's frame
  std::vector<uint32_t> em4;     // parallel to s4: bit b = box b of the task reads the entry
  auto add_task = [&](int32_t I0, int32_t m, int64_t box) {
    int64_t nsrc = 0;
    for (auto& so : sl) nsrc += so.first.y;
    for (int32_t r0 = 0; r0 < m; r0 += rows_cap) {
      const int32_t s0 = (int32_t)s4.size();
      int32_t first = s0, pos = 0;
      for (auto& so : sl)
        for (int32_t p0 = 0; p0 < so.first.y; p0 += kTileCap) {
          const int32_t np = std::min(kTileCap, so.first.y - p0);
          if (pos + np > kTileCap) {
            s4[first].w = (int32_t)s4.size();
            first = (int32_t)s4.size();
            pos = 0;
          }
          s4.push_back(make_int4(so.first.x + p0, np, pos, 0));
          o4.push_back(so.second);
          em4.push_back(~0u);
          pos += np;
        }
      if ((int32_t)s4.size() > first) s4[first].w = (int32_t)s4.size();
      const int32_t mr = std::min(rows_cap, m - r0);
      t4.push_back(make_int4(I0 + r0, mr, s0, (int32_t)s4.size()));
      tbox_of.push_back(box);
      P.packed_pairs += (int64_t)mr * nsrc;
    }
  };
  // Tensor-core tiles hold 128 target rows whatever a task's size: consecutive
  // tasks [a, b) of one pass at level l whose boxes share their ancestor two
  // levels up (so every offset below stays an exact small multiple of h_l) are
  // packed into one task of at most 128 rows and 32 boxes. Its frame is the
  // first box's; each box keeps a record (first row, offset into the frame);
  // its sources are the union of the boxes' sources, moved into the frame, each
  // with the mask of the boxes that read it (the kernel zeroes the other
  // entries of the tile). Returns the new end of the pass.
  auto pack_tasks = [&](int64_t a, int64_t b, int l) -> int64_t {
    std::vector<int4> mt;
    std::vector<int2> mtb;
    const double hl = P.h_box[l];
    for (int64_t i = a; i < b;) {
      int64_t j = i + 1;
      int32_t rows = t4[i].y;
      const uint64_t anc = l >= 2 ? h->lv[l].h_bkey[tbox_of[i]] >> (2 * d) : 0;
      while (j < b && j - i < 32 && t4[j].x == t4[j - 1].x + t4[j - 1].y && rows + t4[j].y <= 128 &&
             (l < 2 || (h->lv[l].h_bkey[tbox_of[j]] >> (2 * d)) == anc)) {
        rows += t4[j].y;
        ++j;
      }
      const int32_t r0 = (int32_t)brow4.size();
      if (j == i + 1) {
        mt.push_back(t4[i]);
        brow4.push_back(0);
        boff4.push_back(make_float4(0.f, 0.f, 0.f, 0.f));
        mtb.push_back(make_int2(r0, 1));
        i = j;
        continue;
      }
      int64_t cf[kMaxDim], cb[kMaxDim];
      coords(l, tbox_of[i], cf);
      const int32_t e0 = (int32_t)s4.size();
      std::vector<std::pair<int32_t, int32_t>> seen;  // (source start, entry index)
      for (int64_t k = i; k < j; ++k) {
        coords(l, tbox_of[k], cb);
        float bo[4] = {0.f, 0.f, 0.f, 0.f};
        for (int q = 0; q < d && q < 4; ++q) bo[q] = (float)((double)(cb[q] - cf[q]) * hl);
        brow4.push_back(t4[k].x - t4[i].x);
        boff4.push_back(make_float4(bo[0], bo[1], bo[2], bo[3]));
        const uint32_t bit = 1u << (uint32_t)(k - i);
        for (int32_t e = t4[k].z; e < t4[k].w; ++e) {
          const int4 se = s4[e];
          int32_t at = -1;
          for (const auto& sv : seen)
            if (sv.first == se.x) {
              at = sv.second;
              break;
            }
          if (at < 0) {
            // the entry's box offset from box k (an integer times h_l), then from the frame
            const float4 of = o4[e];
            const float ov[4] = {of.x, of.y, of.z, of.w};
            float nv[4] = {0.f, 0.f, 0.f, 0.f};
            for (int q = 0; q < d && q < 4; ++q)
              nv[q] = (float)((std::nearbyint((double)ov[q] / hl) + (double)(cb[q] - cf[q])) * hl);
            at = (int32_t)s4.size();
            s4.push_back(make_int4(se.x, se.y, 0, 0));
            o4.push_back(make_float4(nv[0], nv[1], nv[2], nv[3]));
            em4.push_back(0u);
            seen.push_back({se.x, at});
          }
          em4[at] |= bit;
        }
      }
      mt.push_back(make_int4(t4[i].x, rows, e0, (int32_t)s4.size()));
      mtb.push_back(make_int2(r0, (int32_t)(j - i)));
      i = j;
    }
    t4.resize(a);
    tbox_of.resize(a);
    tb4.resize(a);
    for (size_t q = 0; q < mt.size(); ++q) {
      t4.push_back(mt[q]);
      tbox_of.push_back(-1);
      tb4.push_back(mtb[q]);
    }
    return (int64_t)t4.size();
  };
  auto box_src = [&](int l, int64_t I, int64_t J) {  // source box J in target box I's frame
    const Level& L = h->lv[l];
    int64_t cI[kMaxDim], cJ[kMaxDim];
    coords(l, I, cI);
    coords(l, J, cJ);
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < d && k < 4; ++k) v[k] = (float)((double)(cJ[k] - cI[k]) * P.h_box[l]);
    sl.push_back({make_int2(L.h_bstart[J], L.h_bstart[J + 1] - L.h_bstart[J]), make_float4(v[0], v[1], v[2], v[3])});
    need4[l] = 1;
  };
  // tasks of one launch in decreasing order of their pairs: the hardware
  // hands CTAs out in order, so the long tasks start first (each task owns
  // its rows, so the order changes no sum)
  auto sort_tasks = [&](int64_t a, int64_t b) {
    if (!tc_tiles) return;  // the CUDA-core tiles keep tree order (they run beside the applies)
    // a tensor-core tile costs its 128 rows whatever the task's rows
    std::vector<std::pair<int64_t, int64_t>> w;
    w.reserve((size_t)(b - a));
    for (int64_t t = a; t < b; ++t) {
      int64_t n = 0;
      for (int32_t e = t4[t].z; e < t4[t].w; ++e) n += s4[e].y;
      w.push_back({-(int64_t)((t4[t].y + 127) / 128) * n, t});
    }
    std::stable_sort(w.begin(), w.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    std::vector<int4> ts((size_t)(b - a));
    std::vector<int2> tbs((size_t)(b - a));
    for (int64_t t = a; t < b; ++t) {
      ts[(size_t)(t - a)] = t4[w[(size_t)(t - a)].second];
      tbs[(size_t)(t - a)] = tb4[w[(size_t)(t - a)].second];
    }
    for (int64_t t = a; t < b; ++t) {
      t4[t] = ts[(size_t)(t - a)];
      tb4[t] = tbs[(size_t)(t - a)];
    }
  };
  P.coarse4.clear();
  // packed tasks: the FP32 tiles, and the float-float near field of FP64 handles
  const bool ffnear = f64 && h->opt.fp64_near == 1;
  if ((!f64 || ffnear) && d <= 4) {
    for (int l = 1; l < h->kappa; ++l) {
      const Level& L = h->lv[l];
      DenseLevel DL;
      DL.level = l;
      DL.t0 = (int64_t)t4.size();
      for (int64_t i = 0; i < L.nb; ++i) {
        sl.clear();
        const int64_t b0 = h->h_blk_off[l] + L.h_iloff[i], b1 = h->h_blk_off[l] + L.h_iloff[i + 1];
        for (int64_t b = b0; b < b1; ++b)
          if (h->h_dense[b]) box_src(l, i, h->h_bsj[b]);
        if (!sl.empty()) add_task(L.h_bstart[i], L.h_bstart[i + 1] - L.h_bstart[i], i);
      }
      DL.t1 = tc_tiles ? pack_tasks(DL.t0, (int64_t)t4.size(), l) : (int64_t)t4.size();
      sort_tasks(DL.t0, DL.t1);
      if (DL.t1 > DL.t0) P.coarse4.push_back(DL);
    }
    // leaf level: tiles per parent box, or lists per leaf box, by work
    const int lk = h->kappa;
    const Level& LK = h->lv[lk];
    int64_t list_pairs = 0, excl_pairs = 0, tile_pairs = 0;
    for (int64_t i = 0; i < LK.nb; ++i) {
      const int64_t m = LK.h_bstart[i + 1] - LK.h_bstart[i];
      for (int32_t e = h->h_nearoff[i]; e < h->h_nearoff[i + 1]; ++e) {
        const int64_t J = h->h_nearidx[e];
        list_pairs += m * (LK.h_bstart[J + 1] - LK.h_bstart[J]);
      }
      if (lk >= 1) {
        const int64_t b0 = h->h_blk_off[lk] + LK.h_iloff[i], b1 = h->h_blk_off[lk] + LK.h_iloff[i + 1];
        for (int64_t b = b0; b < b1; ++b) (h->h_dense[b] ? list_pairs : excl_pairs) += m * h->h_bn[b];
      }
    }
    // neighbours of parent boxes sharing a face of dimension > amax (non-admissible), and the box itself
    std::vector<std::vector<int64_t>> nbr;
    if (lk >= 1) {
      const int lp = lk - 1;
      const Level& LP = h->lv[lp];
      nbr.resize(LP.nb);
      const int64_t side = int64_t(1) << lp;
      int64_t nd = 1;
      for (int k = 0; k < d; ++k) nd *= 3;
      for (int64_t pb = 0; pb < LP.nb; ++pb) {
        int64_t c[kMaxDim], q[kMaxDim];
        coords(lp, pb, c);
        for (int64_t code = 0; code < nd; ++code) {
          int64_t t = code;
          bool inside = true;
          int zeros = 0;
          for (int k = 0; k < d; ++k) {
            const int64_t delta = t % 3 - 1;
            t /= 3;
            q[k] = c[k] + delta;
            zeros += delta == 0;
            inside &= q[k] >= 0 && q[k] < side;
          }
          if (!inside || zeros <= h->opt.admissible_face_dim) continue;  // non-admissible neighbours and itself
          uint64_t key = 0;
          for (int bit = 0; bit < lp; ++bit)
            for (int k = 0; k < d; ++k) key |= (uint64_t)((q[k] >> bit) & 1) << (d * bit + k);
          const auto it = std::lower_bound(LP.h_bkey.begin(), LP.h_bkey.begin() + LP.nb, key);
          if (it != LP.h_bkey.begin() + LP.nb && *it == key) nbr[pb].push_back(it - LP.h_bkey.begin());
        }
        std::sort(nbr[pb].begin(), nbr[pb].end());
        int64_t nsrc = 0;
        for (int64_t qb : nbr[pb]) nsrc += LP.h_bstart[qb + 1] - LP.h_bstart[qb];
        tile_pairs += (int64_t)(LP.h_bstart[pb + 1] - LP.h_bstart[pb]) * nsrc;
      }
    }
    const int mode = h->opt.near_mode;
    P.tiles = lk >= 1 && (mode == 1 || (mode == 0 && (double)(tile_pairs + excl_pairs) <= 1.25 * (double)list_pairs));
    if (P.tiles) {
      // subtract the low-rank (or zero-rank) leaf IL blocks the tiles include
      P.excl4.level = lk;
      P.excl4.t0 = (int64_t)t4.size();
      for (int64_t i = 0; i < LK.nb; ++i) {
        sl.clear();
        const int64_t b0 = h->h_blk_off[lk] + LK.h_iloff[i], b1 = h->h_blk_off[lk] + LK.h_iloff[i + 1];
        for (int64_t b = b0; b < b1; ++b)
          if (!h->h_dense[b]) box_src(lk, i, h->h_bsj[b]);
        if (!sl.empty()) add_task(LK.h_bstart[i], LK.h_bstart[i + 1] - LK.h_bstart[i], i);
      }
      P.excl4.t1 = tc_tiles ? pack_tasks(P.excl4.t0, (int64_t)t4.size(), lk) : (int64_t)t4.size();
      sort_tasks(P.excl4.t0, P.excl4.t1);
      const int lp = lk - 1;
      const Level& LP = h->lv[lp];
      P.leaf4.level = lp;
      P.leaf4.t0 = (int64_t)t4.size();
      for (int64_t pb = 0; pb < LP.nb; ++pb) {
        sl.clear();
        for (int64_t qb : nbr[pb]) box_src(lp, pb, qb);
        add_task(LP.h_bstart[pb], LP.h_bstart[pb + 1] - LP.h_bstart[pb], pb);
      }
      P.leaf4.t1 = tc_tiles ? pack_tasks(P.leaf4.t0, (int64_t)t4.size(), lp) : (int64_t)t4.size();
      sort_tasks(P.leaf4.t0, P.leaf4.t1);
    } else {
      P.excl4 = DenseLevel{lk, 0, 0};
      P.leaf4.level = lk;
      P.leaf4.t0 = (int64_t)t4.size();
      for (int64_t i = 0; i < LK.nb; ++i) {
        sl.clear();
        for (int32_t e = h->h_nearoff[i]; e < h->h_nearoff[i + 1]; ++e) box_src(lk, i, h->h_nearidx[e]);
        if (lk >= 1) {
          const int64_t b0 = h->h_blk_off[lk] + LK.h_iloff[i], b1 = h->h_blk_off[lk] + LK.h_iloff[i + 1];
          for (int64_t b = b0; b < b1; ++b)
            if (h->h_dense[b]) box_src(lk, i, h->h_bsj[b]);
        }
        add_task(LK.h_bstart[i], LK.h_bstart[i + 1] - LK.h_bstart[i], i);
      }
      P.leaf4.t1 = tc_tiles ? pack_tasks(P.leaf4.t0, (int64_t)t4.size(), lk) : (int64_t)t4.size();
      sort_tasks(P.leaf4.t0, P.leaf4.t1);
    }
    if ((int64_t)s4.size() >= INT32_MAX) {
      set_error("packed source list too long");
      return HODLRDD_ERR_UNSUPPORTED;
    }
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
    if (d <= 4) {
      P.hi4.clear();
      P.lo4.clear();
      P.hi4.resize(h->kappa + 1);
      P.lo4.resize(h->kappa + 1);
      for (int l = 0; l <= h->kappa; ++l) {
        if (!need4[l]) continue;
        HD_TRY(P.hi4[l].alloc(h->N));
        HD_TRY(P.lo4[l].alloc(h->N));
        HD_TRY(launch_relhilo(h, l, P.hi4[l].p, P.lo4[l].p, dlo.p, st));
      }
      HD_TRY(upload(P.tasks4, t4, st));
      HD_TRY(upload(P.srcs4, s4, st));
      HD_TRY(upload(P.soff4, o4, st));
      P.tbox4.release();
      P.brow4.release();
      P.boff4.release();
      P.emask4.release();
      if (tc_tiles && !t4.empty()) {
        HD_TRY(upload(P.tbox4, tb4, st));
        HD_TRY(upload(P.brow4, brow4, st));
        HD_TRY(upload(P.boff4, boff4, st));
        HD_TRY(upload(P.emask4, em4, st));
      }
    }
    HD_CUDA(cudaStreamSynchronize(st));
  }
  if (ffnear && d <= 4) {
    std::vector<double> hlo(h->lo, h->lo + d);
    DevBuf<double> dlo;
    HD_TRY(upload(dlo, hlo, st));
    P.hq4.clear();
    P.lq4.clear();
    for (int l = 0; l <= h->kappa; ++l)
      if (need4[l]) HD_TRY(build_ffcoords(h, l, dlo.p, st));
    HD_TRY(upload(P.tasks4, t4, st));
    HD_TRY(upload(P.srcs4, s4, st));
    HD_TRY(upload(P.soff4, o4, st));
    HD_CUDA(cudaStreamSynchronize(st));
  }
  HD_CUDA(cudaStreamSynchronize(st));
  return HODLRDD_OK;
}

// y_l slices the U-applies write: one per level, two with the FP16 tail.
int level_slices(const hodlrdd_s* h) {
  return h->kappa * (h->opt.precision == HODLRDD_PREC_FP32_FP16 ? 2 : 1);
}

int alloc_workspace(hodlrdd_s* h) {
  if (h->opt.precision == HODLRDD_PREC_FP16X2) {
    // chunks of kTcR right-hand sides: x_t, t, the level slices and the near
    // field hold kTcR values per row; the partial sums of cut U panels are
    // followed by the kTcR column maxima of |x_t|
    h->wnr = kTcR;
    HD_TRY(h->xt.alloc((size_t)h->N * kTcR * 4));
    HD_TRY(h->tbuf.alloc((size_t)std::max<int64_t>(h->total_rank, 1) * kTcR * 4));
    HD_TRY(h->ylev.alloc((size_t)std::max(h->kappa, 1) * h->N * kTcR * 4));
    HD_TRY(h->pbuf.alloc(((size_t)std::max<int64_t>(h->plan.tc_parts, 1) * 128 + 1) * kTcR * 4));
    HD_TRY(h->ynear.alloc((size_t)h->N * kTcR));
    HD_TRY(h->err.alloc(1));
    HD_CUDA(cudaMemsetAsync(h->err.p, 0, sizeof(int32_t), h->st));
    HD_CUDA(cudaStreamSynchronize(h->st));
    return HODLRDD_OK;
  }
  // chunks of up to 16 right-hand sides (FP32 with the packed near field)
  // when the caller asked for more than 8, else up to 8
  const int nr = h->opt.max_nrhs >= 16 && h->opt.precision == HODLRDD_PREC_FP32 && h->d <= 4 ? 16 : 8;
  h->wnr = nr;
  const size_t acc = h->opt.precision == HODLRDD_PREC_FP64 ? 8 : 4;
  HD_TRY(h->xt.alloc(((size_t)h->N + 2 * kGuard) * nr * acc));
  HD_TRY(h->tbuf.alloc(((size_t)h->total_rank + 2 * kGuard) * nr * acc));
  HD_TRY(h->ylev.alloc((size_t)std::max(level_slices(h), 1) * h->N * nr * acc));
  // the FP16 tail streams run beside the FP32 ones: their partial sums follow
  const int64_t prows = std::max<int64_t>({h->plan.vs.part_rows, h->plan.us.part_rows, 1}) +
                        std::max<int64_t>(h->plan.vs2.part_rows, h->plan.us2.part_rows);
  HD_TRY(h->pbuf.alloc((size_t)prows * nr * acc));
  if (h->plan.tasks4.n > 0) {
    HD_TRY(h->ynear.alloc((size_t)h->N * nr));
    HD_TRY(h->nctr.alloc(1));
  }
  HD_TRY(h->err.alloc(1));
  HD_CUDA(cudaMemsetAsync(h->xt.p, 0, h->xt.bytes(), h->st));
  HD_CUDA(cudaMemsetAsync(h->tbuf.p, 0, h->tbuf.bytes(), h->st));
  HD_CUDA(cudaMemsetAsync(h->err.p, 0, sizeof(int32_t), h->st));
  HD_CUDA(cudaStreamSynchronize(h->st));
  return HODLRDD_OK;
}

namespace {

// Tracing: take 5 events for one chunk from the handle's pool.
int chunk_events(hodlrdd_s* h, cudaEvent_t* ev, int n) {
  for (int i = 0; i < n; ++i) {
    if (h->ev_pool.empty()) {
      cudaEvent_t e;
      HD_CUDA(cudaEventCreate(&e));
      h->ev_pool.push_back(e);
    }
    ev[i] = h->ev_pool.back();
    h->ev_pool.pop_back();
  }
  h->ev_pending.emplace_back(ev, ev + n);
  return HODLRDD_OK;
}

template <class Acc, class IO, int NR, int D, bool F64>
int launch_dense(hodlrdd_s* h, cudaStream_t st, int sms, const Acc* xt, Acc* yl, IO* y, int ldy, int c0) {
  const Plan& P = h->plan;
  (void)sms;
  // one CTA per task (the hardware scheduler balances tasks of unequal size)
  auto grid_tasks = [](int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(n, 1 << 30)); };
  const double kc = kernel_const(h->K);
  for (const DenseLevel& DL : P.coarse) {
    const float* rel = F64 ? nullptr : P.rel[DL.level].p;
    k_dense<Acc, IO, NR, D, F64, false><<<grid_tasks(DL.t1 - DL.t0), 256, 0, st>>>(
        P.tasks.p, DL.t0, DL.t1, P.srcs.p, P.soff.p, rel, h->pts64.p, h->N, h->d, h->K.id, kc, h->K.scale,
        h->K.diag, xt, yl + (int64_t)(DL.level - 1) * h->N * NR, yl, h->kappa, h->perm.p, y, ldy, c0);
    h->launches += 1;
  }
  const float* rel = F64 ? nullptr : P.rel[h->kappa].p;
  k_dense<Acc, IO, NR, D, F64, true><<<grid_tasks(P.leaf.t1 - P.leaf.t0), 256, 0, st>>>(
      P.tasks.p, P.leaf.t0, P.leaf.t1, P.srcs.p, P.soff.p, rel, h->pts64.p, h->N, h->d, h->K.id, kc, h->K.scale,
      h->K.diag, xt, nullptr, yl, level_slices(h), h->perm.p, y, ldy, c0);
  h->launches += 1;
  HD_CUDA(cudaGetLastError());
  return HODLRDD_OK;
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
  cudaEvent_t ev[7];
  const bool prof = h->profiling;
  // packed near field: one right-hand side in d <= 3 (kernel-specialised
  // tiles), else FP32 multi-RHS tiles for d <= 4
  const bool packed1 = !F64 && NR == 1 && ldx == 1 && c0 == 0 && h->d <= 3 && P.tasks4.n > 0;
  // the near field on SMs of its own (option near_sms): apply CTAs and near
  // CTAs each reserve a whole SM's shared memory, so neither shares an SM
  const int nsplit = packed1 && apply_sms(h, sms) < sms ? split_passes(h) : 0;
  const bool split = nsplit > 0 && nsplit <= std::min(kSplitMaxPass, h->wnr);
  const bool packed = !F64 && h->d <= 4 && P.tasks4.n > 0;
  // FP64, one right-hand side: the float-float near field on the FP32 pipes (option fp64_near)
  const bool ffn = F64 && NR == 1 && h->opt.fp64_near == 1 && P.tasks4.n > 0 && !P.hq4.empty();
  double* ynear64 = reinterpret_cast<double*>(h->ynear.p);  // N doubles fit in the N x 8 floats
  if (prof) {
    HD_TRY(chunk_events(h, ev, (packed || ffn) ? 7 : 5));  // 5, 6: the near field on the aux stream
    HD_CUDA(cudaEventRecord(ev[0], st));
  }
  k_gather<Acc, IO, NR><<<(int)std::min<int64_t>((h->N + 255) / 256, sms * 16), 256, 0, st>>>(x, h->perm.p, h->N,
                                                                                              ldx, c0, xt);
  h->launches += 1;
  if (prof) HD_CUDA(cudaEventRecord(ev[1], st));
  // the near field needs only x_t: on the packed path it runs on the aux
  // stream beside the low-rank applies (HBM-bound against instruction-bound)
  // and joins before the final sum; it is enqueued after the V-apply so that
  // the persistent panel CTAs are placed first
  if (packed || ffn) HD_CUDA(cudaEventRecord(h->ev_fork, st));
  auto fork_near = [&]() -> int {
    if (!packed && !ffn) return HODLRDD_OK;
    HD_CUDA(cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
    if (prof) HD_CUDA(cudaEventRecord(ev[5], h->aux));
    if constexpr (!F64) {
      if (split) HD_TRY(launch_tiles_split(h, h->aux, reinterpret_cast<const float*>(xt)));
      else if (packed1) launch_tiles(h, h->aux, reinterpret_cast<const float*>(xt));
      else HD_TRY(launch_tiles_nr(h, h->aux, reinterpret_cast<const float*>(xt), NR));
    } else {
      HD_TRY(launch_tiles_ff(h, h->aux, reinterpret_cast<const double*>(xt), ynear64));
    }
    if (prof) HD_CUDA(cudaEventRecord(ev[6], h->aux));
    HD_CUDA(cudaEventRecord(h->ev_join, h->aux));
    return HODLRDD_OK;
  };
  using C = PanelCfg<T, NR>;
  const float* sa = Fac<T>::scaled ? h->sv.p : nullptr;
  const float* sb = Fac<T>::scaled ? h->su.p : nullptr;
  Acc* pb = reinterpret_cast<Acc*>(h->pbuf.p);
  const bool skel = h->opt.lowrank_form == 1;
  if (skel && NR != 1) {
    set_error("matvec: the skeleton form applies one right-hand side at a time");
    return HODLRDD_ERR_UNSUPPORTED;
  }
  const bool mixed = h->opt.precision == HODLRDD_PREC_FP32_FP16;
  Acc* pb2 = pb + (size_t)std::max<int64_t>({P.vs.part_rows, P.us.part_rows, 1}) * NR;
  auto args = [&](const Stream& S, const Acc* vec, Acc* out, const int32_t* map, const float* scl, Acc* part) {
    return PanelArgs<T>{reinterpret_cast<const T*>(S.data.p), S.panels.p, S.stages.p, S.cta.p, S.ctas, vec, out, map,
                        scl, part};
  };
  auto args16 = [&](const Stream& S, const float* vec, float* out, const int32_t* map, const float* scl,
                    float* part) {
    return PanelArgs<__half>{reinterpret_cast<const __half*>(S.data.p), S.panels.p, S.stages.p, S.cta.p, S.ctas, vec,
                             out, map, scl, part};
  };
  // one apply stage: uniform storage, or (mixed) the FP32 and FP16 streams in one launch
  auto stage = [&](bool vmode, const Acc* vec, Acc* out) -> int {
    const Stream& S1 = vmode ? P.vs : P.us;
    const Stream& S2 = vmode ? P.vs2 : P.us2;
    const int32_t* m1 = vmode ? P.vmap.p : nullptr;
    const int32_t* m2 = vmode ? P.vmap2.p : nullptr;
    const float* a1 = vmode ? sa : nullptr;
    const float* b1 = vmode ? sb : nullptr;
    bool launched = false;
    if constexpr (std::is_same<T, float>::value && NR <= 8) {
      if (mixed && (S1.ctas > 0 || S2.ctas > 0)) {
        const int grid = std::max(S1.ctas, S2.ctas);
        const PanelArgs<float> A = args(S1, vec, out, m1, nullptr, pb);
        const PanelArgs<__half> B = args16(S2, vec, out, m2, vmode ? P.vscl2.p : nullptr, pb2);
        constexpr int NW = C::kStagesWide, N3 = C::kStagesN;
        bool wide = false;
        if constexpr (NR == 1) {
          if (split) {  // the whole SM's shared memory (near field on SMs of its own), four ring slots
            if (vmode) k_panel_mix<NR, true, NW><<<grid, kSegThreads, panel_smem_full(), st>>>(A, B, h->err.p);
            else k_panel_mix<NR, false, NW><<<grid, kSegThreads, panel_smem_full(), st>>>(A, B, h->err.p);
            wide = true;
          }
        }
        if (!wide) {
          if (vmode) k_panel_mix<NR, true, N3><<<grid, kSegThreads, C::kSmem, st>>>(A, B, h->err.p);
          else k_panel_mix<NR, false, N3><<<grid, kSegThreads, C::kSmem, st>>>(A, B, h->err.p);
        }
        h->launches += 1;
        launched = true;
      }
    }
    if (!launched && S1.ctas > 0 && !S1.h_stages.empty()) {
      const PanelArgs<T> A = args(S1, vec, out, m1, vmode && Fac<T>::scaled ? P.vscl.p : nullptr, pb);
      constexpr int NW = C::kStagesWide, N3 = C::kStagesN;
      bool wide = false;
      if constexpr (NR == 1) {
        if (split) {
          if (vmode) k_panel<T, NR, true, NW><<<S1.ctas, kSegThreads, panel_smem_full(), st>>>(A, h->err.p);
          else k_panel<T, NR, false, NW><<<S1.ctas, kSegThreads, panel_smem_full(), st>>>(A, h->err.p);
          wide = true;
        }
      }
      if (!wide) {
        if (vmode) k_panel<T, NR, true, N3><<<S1.ctas, kSegThreads, C::kSmem, st>>>(A, h->err.p);
        else k_panel<T, NR, false, N3><<<S1.ctas, kSegThreads, C::kSmem, st>>>(A, h->err.p);
      }
      h->launches += 1;
    }
    // sums of cut panels, each part from its own partial-sum area
    if (!S1.h_splits.empty()) {
      if (vmode) k_combine<Acc, NR, true><<<(int)S1.h_cwork.size(), 256, 0, st>>>(S1.splits.p, S1.cwork.p, pb, out,
                                                                                   m1, a1, b1);
      else k_combine<Acc, NR, false><<<(int)S1.h_cwork.size(), 256, 0, st>>>(S1.splits.p, S1.cwork.p, pb, out,
                                                                                nullptr, nullptr, nullptr);
      h->launches += 1;
    }
    if (mixed && !S2.h_splits.empty()) {
      if (vmode) k_combine<Acc, NR, true><<<(int)S2.h_cwork.size(), 256, 0, st>>>(S2.splits.p, S2.cwork.p, pb2, out,
                                                                                   m2, h->sv.p, h->su.p);
      else k_combine<Acc, NR, false><<<(int)S2.h_cwork.size(), 256, 0, st>>>(S2.splits.p, S2.cwork.p, pb2, out,
                                                                                nullptr, nullptr, nullptr);
      h->launches += 1;
    }
    HD_CUDA(cudaGetLastError());
    return HODLRDD_OK;
  };
  if (h->kappa >= 1) {
    HD_CUDA(cudaMemsetAsync(yl, 0, (size_t)level_slices(h) * h->N * NR * sizeof(Acc), st));
    if (skel) HD_TRY(launch_skeleton_rows(h, st, xt, t));
    else HD_TRY(stage(true, xt, t));
  }
  HD_TRY(fork_near());
  if (prof) HD_CUDA(cudaEventRecord(ev[2], st));
  if (h->kappa >= 1) {
    if (skel) HD_TRY(launch_skeleton_cols(h, st, t, yl));
    else HD_TRY(stage(false, t, yl));
  }
  if (prof) HD_CUDA(cudaEventRecord(ev[3], st));
  if (packed) {
    HD_CUDA(cudaStreamWaitEvent(st, h->ev_join, 0));
    if constexpr (!F64 && std::is_same<IO, float>::value)
      HD_TRY(launch_finish(h, st, reinterpret_cast<const float*>(yl), level_slices(h), y, NR, ldx, c0,
                           split ? nsplit : 1));
  } else if (ffn) {
    HD_CUDA(cudaStreamWaitEvent(st, h->ev_join, 0));
    if constexpr (F64 && std::is_same<IO, double>::value)
      HD_TRY(launch_finish_ff(h, st, ynear64, reinterpret_cast<const double*>(yl), h->kappa >= 1 ? level_slices(h) : 0,
                              y, ldx, c0));
  } else if constexpr (NR <= 8) {
    switch (h->d) {
      case 1: HD_TRY((launch_dense<Acc, IO, NR, 1, F64>(h, st, sms, xt, yl, y, ldx, c0))); break;
      case 2: HD_TRY((launch_dense<Acc, IO, NR, 2, F64>(h, st, sms, xt, yl, y, ldx, c0))); break;
      case 3: HD_TRY((launch_dense<Acc, IO, NR, 3, F64>(h, st, sms, xt, yl, y, ldx, c0))); break;
      case 4: HD_TRY((launch_dense<Acc, IO, NR, 4, F64>(h, st, sms, xt, yl, y, ldx, c0))); break;
      default: HD_TRY((launch_dense<Acc, IO, NR, 0, F64>(h, st, sms, xt, yl, y, ldx, c0))); break;
    }
  } else {
    set_error("matvec: chunks of 16 right-hand sides need the packed near field");
    return HODLRDD_ERR_UNSUPPORTED;
  }
  if (prof) HD_CUDA(cudaEventRecord(ev[4], st));
  HD_CUDA(cudaGetLastError());
  return HODLRDD_OK;
}

// dynamic shared memory up to the whole per-block limit, less the rings'
// mbarriers (launches with the near field on SMs of its own reserve it all)
template <class T, int NR, int NS>
int set_smem_attr_ns() {
  const int smem = (int)panel_smem_full();
  HD_CUDA(cudaFuncSetAttribute(k_panel<T, NR, true, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  HD_CUDA(cudaFuncSetAttribute(k_panel<T, NR, false, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  if constexpr (std::is_same<T, float>::value && NR <= 8) {
    HD_CUDA(cudaFuncSetAttribute(k_panel_mix<NR, true, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    HD_CUDA(cudaFuncSetAttribute(k_panel_mix<NR, false, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  }
  return HODLRDD_OK;
}

template <class T, int NR>
int set_smem_attr_nr() {
  HD_TRY((set_smem_attr_ns<T, NR, PanelCfg<T, NR>::kStagesN>()));
  if constexpr (NR == 1) HD_TRY((set_smem_attr_ns<T, NR, PanelCfg<T, NR>::kStagesWide>()));
  return HODLRDD_OK;
}

template <class T>
int set_smem_attr() {
  static PerDeviceOnce once;
  return once.run([] {
    HD_TRY((set_smem_attr_nr<T, 1>()));
    HD_TRY((set_smem_attr_nr<T, 2>()));
    HD_TRY((set_smem_attr_nr<T, 4>()));
    HD_TRY((set_smem_attr_nr<T, 8>()));
    if constexpr (std::is_same<T, float>::value) HD_TRY((set_smem_attr_nr<T, 16>()));
    return (int)HODLRDD_OK;
  });
}

template <class T, class IO>
int matvec_typed(hodlrdd_s* h, const IO* x, IO* y, int nrhs, cudaStream_t st) {
  HD_TRY(set_smem_attr<T>());
  int c0 = 0;
  if (h->opt.lowrank_form == 1) {  // skeleton form: one right-hand side per pass
    for (; c0 < nrhs; ++c0) HD_TRY((matvec_chunk<T, IO, 1>(h, x, y, nrhs, c0, st)));
    return HODLRDD_OK;
  }
  while (c0 < nrhs) {
    const int rem = nrhs - c0;
    bool wide = false;
    if constexpr (std::is_same<T, float>::value) wide = rem >= 16 && h->wnr >= 16 && h->plan.tasks4.n > 0;
    if (wide) {
      if constexpr (std::is_same<T, float>::value) HD_TRY((matvec_chunk<T, IO, 16>(h, x, y, nrhs, c0, st)));
      c0 += 16;
    } else if (rem >= 8) { HD_TRY((matvec_chunk<T, IO, 8>(h, x, y, nrhs, c0, st))); c0 += 8; }
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
    case HODLRDD_PREC_FP32_FP16:
      return matvec_typed<float, float>(h, static_cast<const float*>(x), static_cast<float*>(y), nrhs, st);
    case HODLRDD_PREC_FP16:
      return matvec_typed<__half, float>(h, static_cast<const float*>(x), static_cast<float*>(y), nrhs, st);
    case HODLRDD_PREC_FP16X2:
      return launch_matvec_tc(h, static_cast<const float*>(x), static_cast<float*>(y), nrhs, st);
    default:
      return matvec_typed<__nv_bfloat16, float>(h, static_cast<const float*>(x), static_cast<float*>(y), nrhs, st);
  }
}

// The apply kernels' CTA ranges over apply_sms CTAs, after near_sms changed.
// No product of the handle may be in flight.
int rebalance_applies(hodlrdd_s* h) {
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  const int ctas = apply_sms(h, sms);
  Plan& P = h->plan;
  const size_t e1 = elem_size(h->opt.precision);
  Stream* streams[4] = {&P.vs, &P.us, &P.vs2, &P.us2};
  for (int i = 0; i < 4; ++i) {
    Stream& S = *streams[i];
    if (S.h_stages.empty()) continue;
    balance_ctas(S, i < 2 ? e1 : 2, ctas);
    HD_TRY(upload(S.cta, S.h_cta, h->st));
  }
  HD_CUDA(cudaStreamSynchronize(h->st));
  return HODLRDD_OK;
}

// Option near_sms = -1: products of a zero vector (the work does not depend on
// the values) timed with the near field beside the applies and on R SMs of its
// own, R from 1/8 to 9/32 of the SMs (the near field's share of the product's
// work on the single-right-hand-side forms); the fastest setting is kept, the
// shared one unless a split is at least 1% faster.
int tune_near_sms(hodlrdd_s* h) {
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  h->opt.near_sms = 1;
  const bool can = apply_sms(h, sms) < sms && h->plan.tasks4.n > 0 && h->kappa >= 1 &&
                   split_passes(h) <= std::min(kSplitMaxPass, h->wnr);
  h->opt.near_sms = 0;
  if (!can) return rebalance_applies(h);
  DevBuf<float> x, y;
  HD_TRY(x.alloc((size_t)h->N));
  HD_TRY(y.alloc((size_t)h->N));
  HD_CUDA(cudaMemsetAsync(x.p, 0, x.bytes(), h->st));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  HD_CUDA(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    HD_CUDA(ce);
  }
  const int64_t launches = h->launches;
  std::vector<int> cand = {0};
  for (int f : {8, 12, 13, 14, 15, 16, 18})  // R = f sms / 64
    cand.push_back(std::max(1, std::min(sms - 1, (f * sms + 32) / 64)));
  double best_ms = 0.0;
  int best = 0;
  int rc = HODLRDD_OK;
  for (size_t c = 0; c < cand.size() && rc == HODLRDD_OK; ++c) {
    h->opt.near_sms = cand[c];
    rc = rebalance_applies(h);
    for (int it = 0; it < 2 && rc == HODLRDD_OK; ++it) rc = launch_matvec(h, x.p, y.p, 1, h->st);
    if (rc != HODLRDD_OK) break;
    cudaEventRecord(e0, h->st);
    for (int it = 0; it < 5 && rc == HODLRDD_OK; ++it) rc = launch_matvec(h, x.p, y.p, 1, h->st);
    cudaEventRecord(e1, h->st);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = HODLRDD_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (c == 0 || ms < best_ms * (best == 0 ? 0.99 : 1.0)) {
      best_ms = ms;
      best = cand[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->launches = launches;
  HD_TRY(rc);
  h->opt.near_sms = best;
  return rebalance_applies(h);
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
    // column k of the block is column h_vcol + k of its source box's panels
    for (int k = 0; k < p; ++k) {
      const int64_t pos = (int64_t)P.h_vcol[b] + k;
      const LPanel& L = P.vs.h_lp[P.h_vpanel[b] + pos / vpanel_width<T>()];
      std::vector<T> buf(n);
      HD_CUDA(cudaMemcpy2D(buf.data(), sizeof(T), reinterpret_cast<const T*>(P.vs.data.p) + L.off + pos % vpanel_width<T>(),
                           (size_t)L.ld * sizeof(T), sizeof(T), n, cudaMemcpyDeviceToHost));
      for (int j = 0; j < n; ++j) V[(size_t)k * n + j] = Fac<T>::to_host(buf[j]) * sv[k];
    }
  }
  if (U) {
    // the box's panels are consecutive; the block's columns start at h_ucol[b]
    for (int r0 = 0; r0 < m; r0 += kPanelRows) {
      const LPanel& Pn = P.us.h_lp[P.h_ugroup[b] + r0 / kPanelRows];
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

// The error word read and cleared on one stream, after the work on it: a
// caller that waits for its own stream only (not the whole device).
int take_error_word(hodlrdd_s* h, cudaStream_t st, int32_t* code) {
  *code = 0;
  if (!h->err.p) return HODLRDD_OK;
  HD_CUDA(cudaMemcpyAsync(code, h->err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  HD_CUDA(cudaStreamSynchronize(st));
  if (*code == 0) return HODLRDD_OK;
  HD_CUDA(cudaMemsetAsync(h->err.p, 0, sizeof(int32_t), st));
  HD_CUDA(cudaStreamSynchronize(st));
  return HODLRDD_OK;
}

int read_error_word(hodlrdd_s* h, int32_t* code) {
  *code = 0;
  if (!h->err.p) return HODLRDD_OK;
  HD_CUDA(cudaDeviceSynchronize());
  HD_CUDA(cudaMemcpy(code, h->err.p, sizeof(int32_t), cudaMemcpyDeviceToHost));
  return HODLRDD_OK;
}

}  // namespace hd
