// Internal declarations shared by the translation units of libhodlrdd.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <utility>
#include <memory>
#include <mutex>
#include <vector>

#include "../../include/hodlrdd.h"

namespace hd {

// ------------------------------------------------------------------ errors ----
void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define HD_CUDA(call)                                                   \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) return ::hd::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define HD_TRY(call)                 \
  do {                               \
    int s_ = (call);                 \
    if (s_ != HODLRDD_OK) return s_; \
  } while (0)

// One-time set-up per device (function attributes such as the dynamic
// shared-memory limit apply to the device current when they are set): run(f)
// calls f once for each device ordinal it is called on, the current one, and
// remembers success.
struct PerDeviceOnce {
  std::mutex mu;
  uint64_t done = 0;  // bit per device ordinal
  template <class F>
  int run(F&& f) {
    int dev = 0;
    HD_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && (done >> dev & 1u)) return HODLRDD_OK;
    const int s = f();
    if (s == HODLRDD_OK && dev >= 0 && dev < 64) done |= uint64_t(1) << dev;
    return s;
  }
};

// Test hook: make the k-th device allocation from now fail (k < 0: never).
void debug_fail_alloc_after(int64_t k);
int64_t debug_aca_pool_bytes();  // test hook: cap on the one-pass ACA pool (-1: none)
int dev_alloc(void** p, size_t bytes);

// Owning device buffer. Frees on destruction; never copied.
template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p; n = o.n;
      o.p = nullptr; o.n = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  int alloc(size_t count) {
    release();
    if (count == 0) return HODLRDD_OK;
    void* q = nullptr;
    int s = dev_alloc(&q, count * sizeof(T));
    if (s != HODLRDD_OK) return s;
    p = static_cast<T*>(q);
    n = count;
    return HODLRDD_OK;
  }
  // An optional scratch: cudaMalloc without the allocation-failure hook (its
  // failure only selects a slower path); false when it could not be had.
  bool try_alloc(size_t count) {
    release();
    if (count == 0) return false;
    void* q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    p = static_cast<T*>(q);
    n = count;
    return true;
  }
  size_t bytes() const { return n * sizeof(T); }
};

template <class T>
int upload(DevBuf<T>& d, const std::vector<T>& h, cudaStream_t st) {
  HD_TRY(d.alloc(h.size()));
  if (!h.empty()) HD_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return HODLRDD_OK;
}

template <class T>
int download(std::vector<T>& h, const T* d, size_t n, cudaStream_t st) {
  h.resize(n);
  if (n) HD_CUDA(cudaMemcpyAsync(h.data(), d, n * sizeof(T), cudaMemcpyDeviceToHost, st));
  return HODLRDD_OK;
}

// ------------------------------------------------------------------ kernel ----
struct KernelSpec {
  int id;
  double scale, diag, p0, p1;
};

constexpr int kMaxDim = 8;
constexpr int kPadRows = 2;  // factor columns are padded to a multiple of this many rows

__host__ __device__ inline int64_t pad_rows(int64_t m) { return (m + kPadRows - 1) / kPadRows * kPadRows; }

// Squared distance and F(s) in FP64 with a fixed operation order. The file
// that evaluates entries for the compression is compiled with contraction off,
// so these round exactly like a plain CPU evaluation of the same formulas.
__device__ __forceinline__ double f64_of_s(int id, double s, double p0) {
  switch (id) {
    case HODLRDD_K_LOG:
      return s == 0.0 ? 0.0 : log(sqrt(s));
    case HODLRDD_K_INV_R:
      return s == 0.0 ? 0.0 : 1.0 / sqrt(s);
    case HODLRDD_K_MATERN32: {
      double a = (1.7320508075688772 * sqrt(s)) / p0;
      return (1.0 + a) * exp(-a);
    }
    case HODLRDD_K_GAUSS:
      return exp(-s / (2.0 * p0 * p0));
    case HODLRDD_K_EXP:
      return exp(-sqrt(s) / p0);
    case HODLRDD_K_INV_R2_4D:
      return s == 0.0 ? 0.0 : -1.0 / (39.47841760435743 * s);
    case HODLRDD_K_R:
      return sqrt(s);
    case HODLRDD_K_SIN:
      return sin(sqrt(s));
    case HODLRDD_K_INV_SQRT1P:
      return 1.0 / sqrt(1.0 + sqrt(s));
  }
  return 0.0;
}

// FP32 evaluation for the mixed-precision near field. `c` is a per-kernel
// precomputed constant (see kernel_const32).
__device__ __forceinline__ float f32_of_s(int id, float s, float c) {
  switch (id) {
    case HODLRDD_K_LOG:
      return s == 0.0f ? 0.0f : 0.5f * logf(s);
    case HODLRDD_K_INV_R:
      return s == 0.0f ? 0.0f : rsqrtf(s);
    case HODLRDD_K_MATERN32: {
      float a = c * sqrtf(s);
      return (1.0f + a) * expf(-a);
    }
    case HODLRDD_K_GAUSS:
      return expf(-c * s);
    case HODLRDD_K_EXP:
      return expf(-c * sqrtf(s));
    case HODLRDD_K_INV_R2_4D:
      return s == 0.0f ? 0.0f : c / s;
    case HODLRDD_K_R:
      return sqrtf(s);
    case HODLRDD_K_SIN:
      return sinf(sqrtf(s));
    case HODLRDD_K_INV_SQRT1P:
      return rsqrtf(1.0f + sqrtf(s));
  }
  return 0.0f;
}

// FP64 evaluation for the FP64 matvec near field: same formulas, contraction
// allowed (this is not used where bitwise agreement with the oracle matters).
__device__ __forceinline__ double f64fast_of_s(int id, double s, double c) {
  switch (id) {
    case HODLRDD_K_LOG:
      return s == 0.0 ? 0.0 : 0.5 * log(s);
    case HODLRDD_K_INV_R:
      return s == 0.0 ? 0.0 : rsqrt(s);
    case HODLRDD_K_MATERN32: {
      double a = c * sqrt(s);
      return (1.0 + a) * exp(-a);
    }
    case HODLRDD_K_GAUSS:
      return exp(-c * s);
    case HODLRDD_K_EXP:
      return exp(-c * sqrt(s));
    case HODLRDD_K_INV_R2_4D:
      return s == 0.0 ? 0.0 : c / s;
    case HODLRDD_K_R:
      return sqrt(s);
    case HODLRDD_K_SIN:
      return sin(sqrt(s));
    case HODLRDD_K_INV_SQRT1P:
      return rsqrt(1.0 + sqrt(s));
  }
  return 0.0;
}

// The constant folded into the matvec evaluators above.
inline double kernel_const(const KernelSpec& k) {
  switch (k.id) {
    case HODLRDD_K_MATERN32: return 1.7320508075688772 / k.p0;
    case HODLRDD_K_GAUSS: return 1.0 / (2.0 * k.p0 * k.p0);
    case HODLRDD_K_EXP: return 1.0 / k.p0;
    case HODLRDD_K_INV_R2_4D: return -1.0 / 39.47841760435743;
    default: return 0.0;
  }
}

// ------------------------------------------------------------------ handle ----
struct Level {
  int64_t nb = 0;
  std::vector<int32_t> h_bstart;  // nb + 1
  std::vector<uint64_t> h_bkey;   // nb
  std::vector<int32_t> h_iloff;   // nb + 1 (levels >= 1)
  std::vector<int32_t> h_ilidx;
  DevBuf<int32_t> bstart;
  DevBuf<uint64_t> bkey;
  DevBuf<int32_t> cfirst;  // nb + 1: first child box at level l + 1
  DevBuf<int32_t> bid;     // per tree-order point: its box at this level (build only)
  DevBuf<int32_t> iloff, ilidx;
};

// One bulk copy into the shared-memory ring: lines [s, s + nseg) of sub-panel
// g. `ng` marks the sub-panel's first stage and `last` its final one.
struct Stage {
  int64_t off;    // element offset in the stream
  int32_t nelem;  // elements copied
  int32_t g;      // sub-panel
  int32_t s;      // first line within the sub-panel
  int32_t nseg;   // lines
  int32_t piece;  // unused (-1)
  int32_t last;   // 1 on the sub-panel's final stage
  int32_t ng;     // 1 on the sub-panel's first stage
  int32_t pad;
};

// A sub-panel of a factor stream: P consecutive lines of ld elements (ld a
// multiple of 16 bytes) whose R leading elements are live. Line k multiplies
// the vector value at index vfirst + k. Outputs w < R go to output row out0 + w
// (U-apply) or to t[map[out0 + w]] (V-apply), or, when the panel was cut into
// several sub-panels, to the partial-sum rows part + w.
struct Panel {
  int64_t off;     // element offset of line 0 in the stream
  int32_t ld;
  int32_t R;
  int32_t P;
  int32_t vfirst;
  int32_t out0;
  int32_t part;    // -1: direct output
};

// A panel cut into nsplit sub-panels: output w = sum_s partial row part + s R + w.
struct Split {
  int32_t part;
  int32_t nsplit;
  int32_t R;
  int32_t out0;
};

// A whole panel as stored (host side, for unpacking): element (k, w) at
// off + k ld + w.
struct LPanel {
  int64_t off;
  int32_t ld;
  int32_t R;
  int32_t lines;
};

// A factor stream with its stage schedule: stages [cta[c], cta[c+1]) belong to
// persistent CTA c; a sub-panel never straddles two CTAs.
struct Stream {
  DevBuf<char> data;
  int64_t elems = 0;
  std::vector<LPanel> h_lp;     // whole panels
  std::vector<Panel> h_panels;  // sub-panels
  std::vector<Stage> h_stages;
  std::vector<int32_t> h_cta;
  std::vector<Split> h_splits;
  std::vector<int2> h_cwork;    // combine work items {split, first output}
  int64_t part_rows = 0;        // partial-sum rows of the cut panels
  DevBuf<Panel> panels;
  DevBuf<Stage> stages;
  DevBuf<int32_t> cta;
  DevBuf<Split> splits;
  DevBuf<int2> cwork;
  int ctas = 0;
};

// On-the-fly dense work: per task a target row range and a list of source
// boxes at the same level; `soff` holds, per source, the exact FP32 offset
// (c_I - c_J) h between the boxes' reference corners.
struct DenseLevel {
  int level = 0;
  int64_t t0 = 0, t1 = 0;  // task range
};

// One task of the skeleton apply: a contiguous range of points (the sources
// of a pivot-row task, the targets of a column task) and a range of a gathered
// pivot list (the targets of a row task, the sources of a column task).
struct SkTask {
  int32_t a0, n;   // contiguous points [a0, a0 + n), tree order
  int32_t r0, r1;  // gathered entries [r0, r1)
  int32_t level;   // tree level of the blocks
  int32_t pout;    // row tasks of a cut group: its first partial sum; else -1
  int32_t pad0, pad1;
};

// Tensor-core form (precision FP16X2). A panel is one 128-row M tile of a
// box's factors, stored as planes of 64-element rows of FP16 (128 bytes, the
// width of one 128-byte-swizzled operand atom): plane (piece, half) holds
// rows [arow + (piece * halves + half) * kstride, + kstride), piece 0 the high
// FP16 part and piece 1 the low part scaled by 2^11, half 0 / 1 the M rows
// 0-63 / 64-127. Row k of a plane multiplies row brow + k of the B operand
// (x_t for V panels, t for U panels; rows >= kvalid are zero).
struct TcPanel {
  int64_t arow;    // first stream row of plane (0, 0)
  int32_t kstride; // rows per plane
  int32_t K;       // rows this panel applies (multiple of 16), from plane row koff
  int32_t koff;    // first plane row applied (sub-panels of a cut U panel)
  int32_t kvalid;  // rows with data, counted from koff
  int32_t halves;  // 1 or 2
  int32_t pieces;  // 2 (high and scaled low part) or 1 (high part only)
  int32_t brow;    // first B row (x_t point or t index) of plane row koff
  int32_t out0;    // V: first V column (column map index); U: first output point
  int32_t mvalid;  // D rows with outputs (<= 128)
  int32_t sbox;    // U: scale bound index of the target box (level, box)
  int32_t slice;   // U: output level slice
  int32_t part;    // U: first partial-sum row block of a cut panel (-1: direct output)
};

// A tensor-core factor stream: FP16 planes, panels and per-CTA panel ranges.
struct TcStream {
  DevBuf<__half> data;
  int64_t rows = 0;                // 64-element rows
  std::vector<TcPanel> h_panels;
  std::vector<int32_t> h_cta;      // panels [cta[c], cta[c + 1]) belong to CTA c
  DevBuf<TcPanel> panels;
  DevBuf<int32_t> cta;
  int ctas = 0;
  alignas(64) unsigned char tmap[128];  // CUtensorMap over the stream (2-D: 64 elements x rows)
};

struct Plan {
  Stream vs, us;                   // V per (level, source box); U per (level, target box)
  DevBuf<int32_t> vmap;            // V panel outputs -> t index
  // mixed FP32 / FP16 storage: the trailing terms of each block in FP16 panels
  // (U outputs to a second set of kappa level slices)
  Stream vs2, us2;
  DevBuf<int32_t> vmap2;
  DevBuf<float> vscl, vscl2;       // per V panel output: su * sv of its t column (16-bit streams)
  int64_t tail_cols = 0;           // columns stored in FP16
  std::vector<int64_t> h_vpanel;   // block -> first whole V panel of its source box (or -1)
  std::vector<int32_t> h_vcol;     // block -> first column within its source box's V panels
  std::vector<int64_t> h_ugroup;   // block -> first whole U panel of its (level, box) (or -1)
  std::vector<int32_t> h_ucol;     // block -> first column within its box's U panels
  DevBuf<int4> tasks;              // {I0, m, src_begin, src_end}
  DevBuf<int2> srcs;               // {J0, n}
  DevBuf<float> soff;              // d per source
  std::vector<DenseLevel> coarse;  // dense IL blocks above the leaf level
  DenseLevel leaf;                 // near field + leaf-level dense IL blocks
  std::vector<DevBuf<float>> rel;  // per level (index l): SoA d x N box-relative FP32 coordinates
  // packed form (FP32 arithmetic, d <= 3, one right-hand side): CTA tasks over
  // box-relative coordinates kept as FP32 hi + lo pairs per level
  DevBuf<int4> tasks4;             // {I0, m, src_begin, src_end}, m <= 256
  DevBuf<int4> srcs4;              // {J0, n, position in its staging chunk, chunk end on a chunk's first entry}
  DevBuf<float4> soff4;            // per source: (c_J - c_I) h_l, exact in FP32
  // tensor-core tiles: small boxes packed into one task (null when not packed)
  DevBuf<int2> tbox4;              // per task: {first box record, boxes}
  DevBuf<int32_t> brow4;           // per record: first row of the box within its task
  DevBuf<float4> boff4;            // per record: the box's offset in the task's frame
  DevBuf<uint32_t> emask4;         // per source entry: boxes of its task that read it
  std::vector<DevBuf<float4>> hi4, lo4;  // per level (where used)
  std::vector<DevBuf<float4>> hq4, lq4;  // FP64 float-float near field: box units, 2^-21 grid + remainder
  std::vector<DenseLevel> coarse4; // dense IL blocks above the leaf level
  DenseLevel leaf4;                // final pass: per parent box (tiles) or per leaf box (lists)
  DenseLevel excl4;                // tiles only: low-rank leaf IL blocks to subtract (level kappa)
  bool tiles = false;              // leaf4 runs over parent tiles at level kappa - 1
  int64_t packed_pairs = 0;        // kernel evaluations of the packed path
  std::vector<double> h_box;       // per level: reference side h'_l (20 significant bits)
  // skeleton form (lowrank_form = 1): pivots and LU factors of K(sigma, tau)
  // per low-rank block, kernel entries evaluated on the fly
  DevBuf<SkTask> sk_rtask;         // K(sigma, J) x(J): per source box, pivot-row group, source chunk
  DevBuf<int4> sk_rsum;            // {r0, r1, first partial, chunks} of row groups cut into chunks
  DevBuf<int4> sk_rows;            // pivot rows grouped by source box: {point, slot, block, 0}
  DevBuf<SkTask> sk_ctask;         // y_l(I) += K(I, tau) w: per target box and row chunk
  DevBuf<int2> sk_cols;            // by slot: {pivot column point, block}
  DevBuf<float4> sk_boff;          // per block: (c_J - c_I) h_l, exact in FP32
  DevBuf<double> sk_lu;            // per block, p' x p' column-major: FP64 form L (lower, with diagonal) and
                                   // U (strict upper); FP32 form W = U^-1 L^-1
  DevBuf<int64_t> sk_luoff;        // per block: first element of its p x p matrix
  DevBuf<int32_t> sk_blist;        // blocks with a non-empty skeleton, for the triangular solves
  DevBuf<int32_t> sk_rank;         // per block: skeleton rank p' <= p (leading ACA terms kept)
  DevBuf<int64_t> sk_toff;         // per block: first slot of its p' values in t
  std::vector<int32_t> h_sk_rank;
  std::vector<int64_t> h_sk_toff;
  DevBuf<char> sk_part;            // partial sums of cut row groups (accumulator type)
  DevBuf<const float4*> sk_hi, sk_lo;  // per level: box-relative coordinates (FP32 form)
  int64_t sk_parts = 0;            // partial sums per product
  int64_t sk_pairs = 0;            // kernel evaluations per product and right-hand side
  int64_t sk_terms = 0;            // sum of the skeleton ranks p'
  int64_t sk_bytes = 0;            // bytes of the skeleton data (LU, pivot lists, offsets, tasks)
  // tensor-core form (precision FP16X2)
  TcStream tcv, tcu;               // V panels per (level, source box, M tile); U per (level, target box, M tile)
  DevBuf<int32_t> tc_vmap;         // V column -> t index
  DevBuf<float> tc_fac;            // per t index: su * sv, folded into t by the V-apply
  DevBuf<float> tc_wbox;           // per (level, target box): power of two >= max |t| / sigma_x over its columns
  DevBuf<int2> tc_split;           // cut U panels: {first partial block, sub-panels}
  std::vector<int2> h_tc_split;
  std::vector<int32_t> h_tc_splitp;  // per split: its panel (output rows, slice)
  DevBuf<int32_t> tc_splitp;
  int64_t tc_parts = 0;            // partial-sum blocks of 128 rows
  int64_t tc_tail_cols = 0;        // columns stored as one FP16 piece
};

}  // namespace hd

struct hodlrdd_s {
  // problem
  int d = 0;
  int64_t N = 0;
  hd::KernelSpec K{};
  int leaf = 0;
  double tol = 0.0;
  hodlrdd_options opt{};
  int device = 0;
  cudaStream_t st = nullptr;  // the handle's own stream (build, staging)
  cudaStream_t aux = nullptr; // second stream: the packed near field runs beside the low-rank applies
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  // tree
  int B = 0, kappa = 0;
  double lo[hd::kMaxDim] = {0};
  double side = 0.0, inv = 0.0;
  std::vector<int32_t> h_perm;
  std::vector<uint64_t> h_skey;
  hd::DevBuf<int32_t> perm;    // tree position -> original index
  hd::DevBuf<uint64_t> skey;
  hd::DevBuf<double> pts64;    // SoA d x N, tree order
  hd::DevBuf<float> pts32;     // SoA d x N, tree order
  std::vector<hd::Level> lv;   // levels 0..kappa
  std::vector<int32_t> h_nearoff, h_nearidx;
  hd::DevBuf<int32_t> nearoff, nearidx;

  // blocks (CSR order over levels 1..kappa)
  int64_t nblk = 0;
  std::vector<int32_t> h_blevel, h_bti, h_bsj, h_bI0, h_bm, h_bJ0, h_bn, h_rank, h_dense;
  std::vector<int64_t> h_blk_off;  // level -> first block (size kappa + 2)
  hd::DevBuf<int32_t> bI0, bm, bJ0, bn, rank, dense;
  hd::DevBuf<int64_t> toff;               // first t column / pivot of each block
  std::vector<int64_t> h_toff;
  hd::DevBuf<int32_t> piv_sigma, piv_tau;  // by toff
  int64_t total_rank = 0, n_rank_capped = 0;

  // factors in the handle's precision (plan.vs / plan.us hold the streams)
  hd::DevBuf<float> su, sv;    // per-column scales (16-bit precisions; 1 otherwise)
  int64_t factor_elems = 0, factor_bytes = 0, dense_pairs = 0;
  hd::Plan plan;

  // matvec workspace (right-hand sides are processed in chunks of at most 8);
  // xt and tbuf carry zero guards of kGuard elements on both sides
  hd::DevBuf<char> xt, tbuf, ylev, xstage, ystage;
  int wnr = 8;                 // right-hand sides per chunk the workspace holds (8 or 16)
  hd::DevBuf<char> pbuf;       // partial sums of cut panels
  hd::DevBuf<float> ynear;     // packed near-field sums (tree order)
  hd::DevBuf<int32_t> nctr;    // task counter of the near field on its own SMs (option near_sms)
  hd::DevBuf<int32_t> err;     // device error word of bounded waits
  std::shared_ptr<void> solve_scratch;  // hodlrdd_solve's buffers when this handle is the inner operator
  bool solve_scratch_f64 = false;

  // tracing: events between matvec stages, resolved by hodlrdd_get_profile
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::vector<cudaEvent_t>> ev_pending;  // per chunk: 5 events on the matvec stream (+ 2 on aux)
  double prof_ms[4] = {0, 0, 0, 0};
  int64_t prof_chunks = 0;
  int64_t launches = 0;

  // stats
  hodlrdd_stats stats{};
};

namespace hd {
// Build stages (tree.cu, aca.cu, apply.cu).
int build_tree(hodlrdd_s* h, const double* dpts);
int build_lists(hodlrdd_s* h);
int build_blocks(hodlrdd_s* h);
int run_aca(hodlrdd_s* h, DevBuf<double>& U64, DevBuf<double>& V64, std::vector<int64_t>& uoff64,
            std::vector<int64_t>& voff64);
int pack_factors(hodlrdd_s* h, const DevBuf<double>& U64, const DevBuf<double>& V64,
                 const std::vector<int64_t>& uoff64, const std::vector<int64_t>& voff64);
int build_plan(hodlrdd_s* h);
int alloc_workspace(hodlrdd_s* h);
int launch_matvec(hodlrdd_s* h, const void* x, void* y, int nrhs, cudaStream_t st);
// The apply kernels' CTA ranges after near_sms changed; near_sms = -1 resolved
// by timed products at the end of the build (apply.cu).
int rebalance_applies(hodlrdd_s* h);
int tune_near_sms(hodlrdd_s* h);
int launch_direct(hodlrdd_s* h, const float* x, float* y, cudaStream_t st);
// Tensor-core form (tcapply.cu).
constexpr int kTcR = 64;          // right-hand sides per chunk (the MMA N)
int pack_tc(hodlrdd_s* h, const DevBuf<double>& U64, const DevBuf<double>& V64, const std::vector<int64_t>& uoff64,
            const std::vector<int64_t>& voff64);
int launch_matvec_tc(hodlrdd_s* h, const float* x, float* y, int nrhs, cudaStream_t st);
int64_t tc_device_bytes(const hodlrdd_s* h);
bool tc_near_supported(const hodlrdd_s* h);
inline bool tc_near_kernel(int kid) { return kid != HODLRDD_K_INV_R && kid != HODLRDD_K_INV_R2_4D; }
int launch_tc_near(hodlrdd_s* h, cudaStream_t st, const float* xt, const unsigned int* colmax);
// Packed tensor-core tasks (small boxes in one tile): null pointers = one box per task.
struct TcPack {
  const int2* tbox;
  const int32_t* brow;
  const float4* boff;
  const uint32_t* emask;
};
inline TcPack tc_pack(const Plan& P) { return TcPack{P.tbox4.p, P.brow4.p, P.boff4.p, P.emask4.p}; }
int launch_tc_near_raw(int d, int kid, cudaStream_t st, int64_t ntask, const int4* tasks, const int4* srcs,
                       const float4* soff, const float4* Hi, const float4* Lo, const float* xt,
                       const unsigned int* colmax, float kc, float* ynear, const int2* tbase, const float2* tsd,
                       TcPack pk, int32_t* err);
// tensor-core applies and combine over an explicit panel set (tcapply.cu)
struct TcLaunch {
  const TcStream* S;
  const float* B;
  const unsigned int* colmax;
  const int32_t* vmap;
  const float* fac;
  const float* wbox;
  float* out;
  float* part;
  int64_t N;
};
int launch_tc_stage(bool vmode, const TcLaunch& L, int32_t* err, cudaStream_t st);
int launch_tc_combine(int64_t nsplit, const int2* split, const int32_t* splitp, const TcPanel* panels,
                      const float* part, int64_t N, float* ylev, cudaStream_t st);
// Panel ranges per CTA, each panel weighed by its bytes plus `fixed` bytes' worth
void tc_schedule_stream(TcStream& S, int ctas, double fixed = 32768.0);
int tc_encode_tmap(TcStream& S);
// Near field (near.cu).
constexpr int kGuard = 16;        // zero elements around xt and t (per right-hand side)
constexpr int kTileThreads = 256; // threads of a near-field tile CTA
constexpr int kTileRows = 256;    // target rows per tile task
constexpr int kTileCap = 1024;    // staged source points per chunk
void launch_tiles(hodlrdd_s* h, cudaStream_t st, const float* xt);
// The packed single-RHS near field on near_sms SMs of their own (k_tile_split):
// kSplitGroups tile groups per CTA, at most kSplitMaxPass passes, pass p
// summing into ynear + p N.
constexpr int kSplitGroups = 3;
constexpr int kSplitMaxPass = 8;
constexpr int kSplitGroupBytes = 2 * kTileCap * 16 + 2 * kTileThreads * 4 + 16;
struct SplitPass {
  int64_t t0, n;  // the pass's tasks [t0, t0 + n) of the packed plan
  const float4* Hi;
  const float4* Lo;
  float scale, diag;
  float* out;
};
struct SplitArgs {
  SplitPass pass[kSplitMaxPass];
  int npass;
  int64_t total;
  int* ctr;
};
int split_passes(const hodlrdd_s* h);
int launch_tiles_split(hodlrdd_s* h, cudaStream_t st, const float* xt);
int launch_tiles_nr(hodlrdd_s* h, cudaStream_t st, const float* xt, int nr, int ldx = 0, int cx = 0);
int launch_finish(hodlrdd_s* h, cudaStream_t st, const float* ylev, int slices, float* y, int nr, int ldy, int c0,
                  int nnear = 1);
int launch_relhilo(hodlrdd_s* h, int l, float4* Hi, float4* Lo, const double* dlo, cudaStream_t st);
// float-float near field of FP64 handles (one right-hand side)
int build_ffcoords(hodlrdd_s* h, int l, const double* dlo, cudaStream_t st);
int launch_tiles_ff(hodlrdd_s* h, cudaStream_t st, const double* xt, double* ynear);
int launch_finish_ff(hodlrdd_s* h, cudaStream_t st, const double* ynear, const double* ylev, int slices, double* y,
                     int ldy, int c0);
int unpack_block(hodlrdd_s* h, int64_t b, double* U, double* V);
// Skeleton form (skeleton.cu).
int build_skeleton(hodlrdd_s* h, const DevBuf<double>& U64, const DevBuf<double>& V64,
                   const std::vector<int64_t>& uoff64, const std::vector<int64_t>& voff64);
int build_skeleton_plan(hodlrdd_s* h);
int launch_skeleton_rows(hodlrdd_s* h, cudaStream_t st, const void* xt, void* t);
int launch_skeleton_cols(hodlrdd_s* h, cudaStream_t st, const void* t, void* ylev);
int read_error_word(hodlrdd_s* h, int32_t* code);
int take_error_word(hodlrdd_s* h, cudaStream_t st, int32_t* code);
int check_device(const hodlrdd_s* h, const char* who);
size_t elem_size(int precision);
}  // namespace hd
