// Batched partial-pivoted ACA of every interaction-list block (a5).
//
// The paper compresses each IL block K(I,J) with ACA (Eq. keq1; Algorithm 1):
// K(I,J) ~ sum_k u_k v_k^T = K(I,tau) U^-1 L^-1 K(sigma,J) (Eq. keq2). The
// rules the paper leaves open are fixed as: first pivot row 0; residual row
// a = A(i*,:) - sum_q u_q(i*) v_q; j* = argmax |a_j| (lowest index on ties); an
// exactly zero residual row is skipped; v_k = a / a_j*; residual column
// u_k = A(:,j*) - sum_q v_q(j*) u_q; ||A_k||_F^2 is updated by
// S += 2 sum_{q<k} (u_q.u_k)(v_q.v_k) + |u_k|^2 |v_k|^2; stop after appending term
// k when |u_k||v_k| <= tol sqrt(S) or k = min(m,n); next row = argmax over unused
// rows of |u_k| (lowest index on ties).
//
// GPU organisation. Blocks are binned by size. Up to 256 rows and columns a warp
// owns a block: lanes stride over rows / columns, and the dot products of the
// norm update run one per lane, each summed in index order, so a warp rounds
// exactly like a sequential FP64 evaluation (this file is compiled with FP
// contraction off). Larger blocks get a whole CTA. Each team keeps its block's
// u_k, v_k in a private scratch slab. One pass computes every block: a team that
// finishes a block reserves room for its factors and pivots in a device pool
// (an atomic bump pointer) and copies them there; the host then lays out the
// block-ordered output and a compaction kernel moves each block's factors into
// it. Blocks that found the pool full (possible only when device memory is
// short) are recomputed by a second pass over those blocks alone, with the same
// arithmetic. No spin-waits: every loop is bounded by min(m, n).
#include <algorithm>
#include <climits>

#include "internal.cuh"

namespace hd {
namespace {

struct AcaArgs {
  const double* pts;  // SoA d x N, tree order
  int64_t N;
  int d;
  int kid;
  double scale, p0, tol;
  int dense_if_cheaper;
  const int8_t* dic_blk;  // per block: the dense-if-cheaper rule applies (null: dense_if_cheaper for all)
  const int32_t *I0, *m, *J0, *n;
  const int32_t* list;  // blocks of this bin, largest first
  int32_t nlist;
  int32_t* counter;     // work counter (zeroed before launch)
  int rcap;
  int64_t slab_elems;   // per team: rcap * (mcap + ncap)
  double* slab;
  // pass 1 outputs
  int32_t* rank;
  int32_t* dense;
  int32_t* capped;
  // pass 2 outputs (null in pass 1)
  double* U64;
  double* V64;
  const int64_t* uoff;
  const int64_t* voff;
  const int64_t* toff;
  int32_t* sig_out;
  int32_t* tau_out;
  int32_t* err;  // set when pass 2 disagrees with pass 1 (nothing is written then)
  // pass 1: the pool (factors k (m + n) doubles, then the 2k pivots as doubles)
  double* pool;
  int64_t pool_elems;
  unsigned long long* pool_top;
  int64_t* poff;  // per block: its place in the pool, -1 when it did not fit
};

__device__ __forceinline__ double entry(const AcaArgs& A, const double* xr, int64_t col) {
  double s = 0.0;
  for (int k = 0; k < A.d; ++k) {
    double t = xr[k] - A.pts[(size_t)k * A.N + col];
    s = s + t * t;
  }
  return A.scale * f64_of_s(A.kid, s, A.p0);
}

struct WarpTeam {
  __device__ int tid() const { return threadIdx.x & 31; }
  __device__ int size() const { return 32; }
  __device__ void sync() const { __syncwarp(); }
  __device__ long long bcast(long long v) const { return __shfl_sync(0xffffffffu, v, 0); }
  __device__ void argmax(double& v, int& i) const {
    for (int o = 16; o; o >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, v, o);
      int oi = __shfl_xor_sync(0xffffffffu, i, o);
      if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
    }
  }
  __device__ int min_int(int v) const {
    for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
  }
  // spu[q] = u_q . u_k and spv[q] = v_q . v_k for q = 0..k (q = k gives the
  // squared norms), each summed in index order by one lane.
  __device__ void dots(const double* Us, const double* Vs, int k, int m, int n, double* spu, double* spv) const {
    for (int q = tid(); q <= k; q += 32) {
      double du = 0.0, dv = 0.0;
      const double* uq = Us + (size_t)q * m;
      const double* uk = Us + (size_t)k * m;
      for (int i = 0; i < m; ++i) du = du + uq[i] * uk[i];
      const double* vq = Vs + (size_t)q * n;
      const double* vk = Vs + (size_t)k * n;
      for (int j = 0; j < n; ++j) dv = dv + vq[j] * vk[j];
      spu[q] = du;
      spv[q] = dv;
    }
    __syncwarp();
  }
};

struct CtaTeam {
  double* red_v;
  int* red_i;
  long long* red_ll;
  __device__ int tid() const { return threadIdx.x; }
  __device__ int size() const { return blockDim.x; }
  __device__ void sync() const { __syncthreads(); }
  __device__ long long bcast(long long v) const {
    if (threadIdx.x == 0) *red_ll = v;
    __syncthreads();
    v = *red_ll;
    __syncthreads();
    return v;
  }
  __device__ void argmax(double& v, int& i) const {
    for (int o = 16; o; o >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, v, o);
      int oi = __shfl_xor_sync(0xffffffffu, i, o);
      if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) { red_v[w] = v; red_i[w] = i; }
    __syncthreads();
    v = red_v[0];
    i = red_i[0];
    for (int q = 1; q < nw; ++q)
      if (red_v[q] > v || (red_v[q] == v && red_i[q] < i)) { v = red_v[q]; i = red_i[q]; }
    __syncthreads();
  }
  __device__ int min_int(int v) const {
    for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) red_i[w] = v;
    __syncthreads();
    v = red_i[0];
    for (int q = 1; q < nw; ++q) v = min(v, red_i[q]);
    __syncthreads();
    return v;
  }
  // One warp per dot product, lanes striding the index, butterfly reduction.
  __device__ void dots(const double* Us, const double* Vs, int k, int m, int n, double* spu, double* spv) const {
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int q = w; q <= k; q += nw) {
      double du = 0.0, dv = 0.0;
      const double* uq = Us + (size_t)q * m;
      const double* uk = Us + (size_t)k * m;
      for (int i = lane; i < m; i += 32) du = du + uq[i] * uk[i];
      const double* vq = Vs + (size_t)q * n;
      const double* vk = Vs + (size_t)k * n;
      for (int j = lane; j < n; j += 32) dv = dv + vq[j] * vk[j];
      for (int o = 16; o; o >>= 1) {
        du = du + __shfl_xor_sync(0xffffffffu, du, o);
        dv = dv + __shfl_xor_sync(0xffffffffu, dv, o);
      }
      if (lane == 0) { spu[q] = du; spv[q] = dv; }
    }
    __syncthreads();
  }
};

// Shared memory of one team.
struct TeamSmem {
  double* sq;   // U[q][i*]   (rcap)
  double* sv;   // V[q][j*]   (rcap)
  double* spu;  // (rcap + 1)
  double* spv;  // (rcap + 1)
  int32_t* sig; // (rcap)
  int32_t* tau; // (rcap)
  uint32_t* used;  // ceil(mcap / 32)
};

__host__ __device__ inline size_t team_smem_bytes(int rcap, int mcap) {
  size_t b = (size_t)(4 * rcap + 2) * sizeof(double) + (size_t)2 * rcap * sizeof(int32_t) +
             (size_t)((mcap + 31) / 32) * sizeof(uint32_t);
  return (b + 15) / 16 * 16;  // keeps every team's doubles 16-byte aligned
}

__device__ inline TeamSmem carve(char* base, int rcap, int mcap) {
  TeamSmem s;
  double* dp = reinterpret_cast<double*>(base);
  s.sq = dp;
  s.sv = dp + rcap;
  s.spu = dp + 2 * rcap;
  s.spv = dp + 3 * rcap + 1;
  int32_t* ip = reinterpret_cast<int32_t*>(dp + 4 * rcap + 2);
  s.sig = ip;
  s.tau = ip + rcap;
  s.used = reinterpret_cast<uint32_t*>(ip + 2 * rcap);
  (void)mcap;
  return s;
}

template <class Team>
__device__ void aca_block(const Team& T, const AcaArgs& A, int32_t b, double* Us, double* Vs, const TeamSmem& S) {
  const int tid = T.tid(), TS = T.size();
  const int32_t I0 = A.I0[b], m = A.m[b], J0 = A.J0[b], n = A.n[b];
  const int kmax = min(m, n);
  const int d = A.d;
  for (int w = tid; w < (m + 31) / 32; w += TS) S.used[w] = 0u;
  T.sync();
  int k = 0, nused = 0, istar = 0;
  double Sf = 0.0;
  bool dense = false, capped = false;
  const bool dic = A.dic_blk ? A.dic_blk[b] != 0 : A.dense_if_cheaper != 0;
  double xr[kMaxDim];
  while (true) {
    for (int c = 0; c < d; ++c) xr[c] = A.pts[(size_t)c * A.N + I0 + istar];
    for (int q = tid; q < k; q += TS) S.sq[q] = Us[(size_t)q * m + istar];
    T.sync();
    // residual row i*
    double best = -1.0;
    int bj = INT_MAX;
    for (int j = tid; j < n; j += TS) {
      double s = 0.0;
      for (int q = 0; q < k; ++q) s = s + S.sq[q] * Vs[(size_t)q * n + j];
      double a = entry(A, xr, (int64_t)J0 + j) - s;
      Vs[(size_t)k * n + j] = a;
      double aa = fabs(a);
      if (aa > best) { best = aa; bj = j; }
    }
    T.argmax(best, bj);
    if (!(best >= 0.0) || bj >= n) {  // no comparable entry (NaN row): apply the block exactly
      dense = true;
      break;
    }
    if (tid == 0) S.used[istar >> 5] |= 1u << (istar & 31);
    ++nused;
    T.sync();
    if (best == 0.0) {  // exactly zero residual row: next unused row
      if (nused == m) break;
      int cand = INT_MAX;
      for (int w = tid; w < (m + 31) / 32; w += TS) {
        uint32_t free_bits = ~S.used[w];
        if (w == (m - 1) / 32 && (m & 31)) free_bits &= (1u << (m & 31)) - 1u;
        if (free_bits) cand = min(cand, w * 32 + __ffs(free_bits) - 1);
      }
      istar = T.min_int(cand);
      continue;
    }
    const double piv = Vs[(size_t)k * n + bj];
    if (tid == 0) { S.sig[k] = istar; S.tau[k] = bj; }
    for (int q = tid; q < k; q += TS) S.sv[q] = Vs[(size_t)q * n + bj];
    T.sync();  // every thread holds piv before row k (and with it the pivot entry) is rescaled
    for (int j = tid; j < n; j += TS) Vs[(size_t)k * n + j] = Vs[(size_t)k * n + j] / piv;
    T.sync();
    // residual column j*
    double xc[kMaxDim];
    for (int c = 0; c < d; ++c) xc[c] = A.pts[(size_t)c * A.N + J0 + bj];
    double ubest = -1.0;
    int ui = INT_MAX;
    for (int i = tid; i < m; i += TS) {
      double s = 0.0;
      for (int q = 0; q < k; ++q) s = s + S.sv[q] * Us[(size_t)q * m + i];
      double u = entry(A, xc, (int64_t)I0 + i) - s;
      Us[(size_t)k * m + i] = u;
      if (!((S.used[i >> 5] >> (i & 31)) & 1u)) {
        double au = fabs(u);
        if (au > ubest) { ubest = au; ui = i; }
      }
    }
    T.argmax(ubest, ui);
    T.sync();
    T.dots(Us, Vs, k, m, n, S.spu, S.spv);
    double cross = 0.0;
    for (int q = 0; q < k; ++q) cross = cross + S.spu[q] * S.spv[q];
    const double uu = S.spu[k], vv = S.spv[k];
    Sf = Sf + 2.0 * cross + uu * vv;
    ++k;
    T.sync();
    if (dic && (int64_t)k * (m + n) >= (int64_t)m * n) { dense = true; break; }
    if (sqrt(uu) * sqrt(vv) <= A.tol * sqrt(fmax(Sf, 0.0))) break;
    if (k == kmax) break;
    if (k == A.rcap) { dense = true; capped = true; break; }
    if (nused == m) break;
    if (ui >= m) {  // no comparable unused row (NaN column): apply the block exactly
      dense = true;
      break;
    }
    istar = ui;
  }
  const int32_t rank_out = dense ? 0 : k;
  if (A.U64 != nullptr) {
    // pass 2: the output was laid out from pass 1's rank; never write past it
    if (rank_out != A.rank[b]) {
      if (tid == 0) atomicExch(A.err, 1);
      T.sync();
      return;
    }
  } else if (tid == 0) {
    A.rank[b] = rank_out;
    A.dense[b] = dense ? 1 : 0;
    A.capped[b] = capped ? 1 : 0;
  }
  if (A.U64 == nullptr && A.pool != nullptr) {
    // one pass: the factors and pivots into the pool, if there is room
    long long off = -1;
    if (rank_out > 0) {
      const long long need = (long long)k * (m + n) + 2LL * k;
      if (tid == 0) {
        const unsigned long long at = atomicAdd(A.pool_top, (unsigned long long)need);
        off = at + (unsigned long long)need <= (unsigned long long)A.pool_elems ? (long long)at : -1LL;
      }
      off = T.bcast(off);
      if (off >= 0) {
        double* P = A.pool + off;
        for (int64_t e = tid; e < (int64_t)k * m; e += TS) P[e] = Us[e];
        for (int64_t e = tid; e < (int64_t)k * n; e += TS) P[(int64_t)k * m + e] = Vs[e];
        for (int q = tid; q < k; q += TS) {
          P[(int64_t)k * (m + n) + q] = (double)S.sig[q];
          P[(int64_t)k * (m + n) + k + q] = (double)S.tau[q];
        }
      }
    }
    if (tid == 0) A.poff[b] = off;
  }
  if (A.U64 != nullptr && !dense && k > 0) {
    double* Uo = A.U64 + A.uoff[b];
    double* Vo = A.V64 + A.voff[b];
    for (int64_t e = tid; e < (int64_t)k * m; e += TS) Uo[e] = Us[e];
    for (int64_t e = tid; e < (int64_t)k * n; e += TS) Vo[e] = Vs[e];
    for (int q = tid; q < k; q += TS) {
      A.sig_out[A.toff[b] + q] = S.sig[q];
      A.tau_out[A.toff[b] + q] = S.tau[q];
    }
  }
  T.sync();
}

__global__ void k_aca_warp(AcaArgs A, int mcap) {
  extern __shared__ __align__(16) char smem[];
  const int team = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int team_id = blockIdx.x * (blockDim.x >> 5) + team;
  TeamSmem S = carve(smem + team * team_smem_bytes(A.rcap, mcap), A.rcap, mcap);
  double* slab = A.slab + (size_t)team_id * A.slab_elems;
  WarpTeam T;
  while (true) {
    int it = 0;
    if (lane == 0) it = atomicAdd(A.counter, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= A.nlist) break;
    const int32_t b = A.list[it];
    double* Us = slab;
    double* Vs = slab + (size_t)A.rcap * A.m[b];
    aca_block(T, A, b, Us, Vs, S);
  }
}

__global__ void k_aca_cta(AcaArgs A, int mcap) {
  extern __shared__ __align__(16) char smem[];
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ long long red_ll;
  __shared__ int s_it;
  TeamSmem S = carve(smem, A.rcap, mcap);
  double* slab = A.slab + (size_t)blockIdx.x * A.slab_elems;
  CtaTeam T{red_v, red_i, &red_ll};
  while (true) {
    if (threadIdx.x == 0) s_it = atomicAdd(A.counter, 1);
    __syncthreads();
    const int it = s_it;
    __syncthreads();
    if (it >= A.nlist) break;
    const int32_t b = A.list[it];
    double* Us = slab;
    double* Vs = slab + (size_t)A.rcap * A.m[b];
    aca_block(T, A, b, Us, Vs, S);
  }
}

// Block-ordered factors and pivots from the pool: one CTA per block (stride).
__global__ void k_aca_compact(int64_t nblk, const int64_t* __restrict__ poff, const int32_t* __restrict__ rank,
                              const int32_t* __restrict__ bm, const int32_t* __restrict__ bn,
                              const double* __restrict__ pool, const int64_t* __restrict__ uoff,
                              const int64_t* __restrict__ voff, const int64_t* __restrict__ toff,
                              double* __restrict__ U64, double* __restrict__ V64, int32_t* __restrict__ sig,
                              int32_t* __restrict__ tau) {
  for (int64_t b = blockIdx.x; b < nblk; b += gridDim.x) {
    const int k = rank[b];
    const int64_t off = poff[b];
    if (k <= 0 || off < 0) continue;
    const int64_t m = bm[b], n = bn[b];
    const double* P = pool + off;
    for (int64_t e = threadIdx.x; e < k * m; e += blockDim.x) U64[uoff[b] + e] = P[e];
    for (int64_t e = threadIdx.x; e < k * n; e += blockDim.x) V64[voff[b] + e] = P[k * m + e];
    for (int q = threadIdx.x; q < k; q += blockDim.x) {
      sig[toff[b] + q] = (int32_t)P[k * (m + n) + q];
      tau[toff[b] + q] = (int32_t)P[k * (m + n) + k + q];
    }
  }
}

struct Bin {
  int lo, hi;       // max(m, n) in (lo, hi]
  bool warp;
  int threads;      // CTA team size
  std::vector<int32_t> list;
  int rcap = 0, mcap = 0, ncap = 0;
  int teams = 0;
  DevBuf<int32_t> dlist, counter;
  DevBuf<double> slab;
  cudaStream_t st = nullptr;
};

}  // namespace

int run_aca(hodlrdd_s* h, DevBuf<double>& U64, DevBuf<double>& V64, std::vector<int64_t>& uoff64,
            std::vector<int64_t>& voff64) {
  const int64_t nblk = h->nblk;
  h->h_rank.assign(nblk, 0);
  h->h_dense.assign(nblk, 0);
  HD_TRY(h->rank.alloc(nblk));
  HD_TRY(h->dense.alloc(nblk));
  DevBuf<int32_t> capped;
  HD_TRY(capped.alloc(nblk));
  uoff64.assign(nblk + 1, 0);
  voff64.assign(nblk + 1, 0);
  if (nblk == 0) {
    h->total_rank = 0;
    HD_TRY(h->toff.alloc(1));
    HD_CUDA(cudaMemsetAsync(h->toff.p, 0, sizeof(int64_t), h->st));
    return HODLRDD_OK;
  }

  Bin bins[4] = {{0, 64, true, 32}, {64, 256, true, 32}, {256, 2048, false, 256}, {2048, INT_MAX, false, 512}};
  for (int64_t b = 0; b < nblk; ++b) {
    int mx = std::max(h->h_bm[b], h->h_bn[b]);
    for (auto& B : bins)
      if (mx > B.lo && mx <= B.hi) { B.list.push_back((int32_t)b); break; }
  }
  int dev_sms = 0;
  HD_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, h->device));
  // dense_if_cheaper 2: the rule holds at the leaf level only, coarser blocks keep their factors
  const int dmode = h->opt.dense_if_cheaper;
  std::vector<int8_t> hdic((size_t)std::max<int64_t>(nblk, 1), 0);
  for (int64_t b = 0; b < nblk; ++b) hdic[b] = dmode == 1 || (dmode == 2 && h->h_blevel[b] == h->kappa) ? 1 : 0;
  DevBuf<int8_t> ddic;
  HD_TRY(upload(ddic, hdic, h->st));
  for (auto& B : bins) {
    if (B.list.empty()) continue;
    std::sort(B.list.begin(), B.list.end(), [&](int32_t a, int32_t c) {
      int64_t sa = (int64_t)h->h_bm[a] * h->h_bn[a], sc = (int64_t)h->h_bm[c] * h->h_bn[c];
      return sa != sc ? sa > sc : a < c;
    });
    for (int32_t b : B.list) {
      int64_t m = h->h_bm[b], n = h->h_bn[b];
      int64_t natural = hdic[b] ? (m * n + (m + n) - 1) / (m + n) : std::min(m, n);
      B.rcap = std::max<int>(B.rcap, (int)natural);
      B.mcap = std::max<int>(B.mcap, (int)m);
      B.ncap = std::max<int>(B.ncap, (int)n);
    }
    if (!B.warp) B.rcap = std::min(B.rcap, std::max(1, h->opt.aca_max_rank));
    B.rcap = std::max(B.rcap, 1);
    const int64_t slab = (int64_t)B.rcap * (B.mcap + B.ncap);
    const int64_t budget = (int64_t)6 << 30;  // bytes of scratch per bin
    int64_t by_mem = std::max<int64_t>(1, budget / (slab * (int64_t)sizeof(double)));
    int64_t resident = B.warp ? (int64_t)dev_sms * 32 : (int64_t)dev_sms * (B.threads == 256 ? 4 : 2);
    B.teams = (int)std::min<int64_t>({(int64_t)B.list.size(), by_mem, resident});
    if (B.warp) B.teams = (B.teams + 3) / 4 * 4;  // 4 warp teams per CTA
    HD_TRY(upload(B.dlist, B.list, h->st));
    HD_TRY(B.counter.alloc(1));
    HD_TRY(B.slab.alloc((size_t)B.teams * slab));
  }
  HD_CUDA(cudaStreamSynchronize(h->st));

  auto launch_all = [&](AcaArgs base) -> int {
    // The largest blocks first, each bin on its own stream so bins overlap.
    cudaEvent_t start_ev;
    HD_CUDA(cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming));
    HD_CUDA(cudaEventRecord(start_ev, h->st));
    int rc = HODLRDD_OK;
    for (int bi = 3; bi >= 0 && rc == HODLRDD_OK; --bi) {
      Bin& B = bins[bi];
      if (B.list.empty()) continue;
      if (!B.st) {
        if (cudaStreamCreateWithFlags(&B.st, cudaStreamNonBlocking) != cudaSuccess) { rc = HODLRDD_ERR_CUDA; break; }
      }
      cudaStreamWaitEvent(B.st, start_ev, 0);
      AcaArgs A = base;
      A.list = B.dlist.p;
      A.nlist = (int32_t)B.list.size();
      A.counter = B.counter.p;
      A.rcap = B.rcap;
      A.slab_elems = (int64_t)B.rcap * (B.mcap + B.ncap);
      A.slab = B.slab.p;
      cudaMemsetAsync(B.counter.p, 0, sizeof(int32_t), B.st);
      size_t sm = team_smem_bytes(B.rcap, B.mcap);
      if (B.warp) {
        size_t total = sm * 4;
        cudaFuncSetAttribute(k_aca_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)total);
        k_aca_warp<<<B.teams / 4, 128, total, B.st>>>(A, B.mcap);
      } else {
        cudaFuncSetAttribute(k_aca_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_aca_cta<<<B.teams, B.threads, sm, B.st>>>(A, B.mcap);
      }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) rc = cuda_fail(e, "ACA launch", __FILE__, __LINE__);
    }
    for (auto& B : bins)
      if (B.st) {
        cudaError_t e = cudaStreamSynchronize(B.st);
        if (e != cudaSuccess && rc == HODLRDD_OK) rc = cuda_fail(e, "ACA kernel", __FILE__, __LINE__);
      }
    cudaEventDestroy(start_ev);
    return rc;
  };

  AcaArgs base{};
  base.pts = h->pts64.p;
  base.N = h->N;
  base.d = h->d;
  base.kid = h->K.id;
  base.scale = h->K.scale;
  base.p0 = h->K.p0;
  base.tol = h->tol;
  base.dense_if_cheaper = dmode == 1 ? 1 : 0;
  base.dic_blk = ddic.p;
  base.I0 = h->bI0.p;
  base.m = h->bm.p;
  base.J0 = h->bJ0.p;
  base.n = h->bn.p;
  base.rank = h->rank.p;
  base.dense = h->dense.p;
  base.capped = capped.p;
  // the pool of the one-pass factors: half of the free device memory beyond a
  // reserve (the block-ordered output needs as much again), at most 128 GB
  DevBuf<double> pool;
  DevBuf<unsigned long long> pool_top;
  DevBuf<int64_t> poff;
  {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      fr = 0;
    }
    const int64_t reserve = (int64_t)2 << 30;
    int64_t bytes = std::min<int64_t>(((int64_t)fr - reserve) / 2, (int64_t)128 << 30);
    if (bytes < ((int64_t)64 << 20)) bytes = 0;
    const int64_t cap = debug_aca_pool_bytes();  // tests: a small pool sends blocks to the second pass
    if (cap >= 0) bytes = std::min(bytes, cap);
    if (bytes >= (int64_t)sizeof(double) && pool.try_alloc((size_t)bytes / sizeof(double)) &&
        pool_top.try_alloc(1) && poff.try_alloc(nblk) &&
        cudaMemsetAsync(pool_top.p, 0, sizeof(unsigned long long), h->st) == cudaSuccess &&
        cudaStreamSynchronize(h->st) == cudaSuccess) {
      base.pool = pool.p;
      base.pool_elems = (int64_t)pool.n;
      base.pool_top = pool_top.p;
      base.poff = poff.p;
    } else {
      cudaGetLastError();
      pool.release();  // two passes: ranks, then the same arithmetic writing the factors
    }
  }
  int rc = launch_all(base);  // ranks (and, with the pool, the factors)
  if (rc == HODLRDD_OK) {
    std::vector<int32_t> hcap;
    std::vector<int64_t> hpoff;
    rc = download(h->h_rank, h->rank.p, nblk, h->st);
    if (rc == HODLRDD_OK) rc = download(h->h_dense, h->dense.p, nblk, h->st);
    if (rc == HODLRDD_OK) rc = download(hcap, capped.p, nblk, h->st);
    if (rc == HODLRDD_OK && base.pool) rc = download(hpoff, poff.p, nblk, h->st);
    if (rc == HODLRDD_OK && cudaStreamSynchronize(h->st) != cudaSuccess) rc = HODLRDD_ERR_CUDA;
    if (rc == HODLRDD_OK) {
      std::vector<int64_t> toff(nblk + 1, 0);
      h->n_rank_capped = 0;
      for (int64_t b = 0; b < nblk; ++b) {
        uoff64[b + 1] = uoff64[b] + (int64_t)h->h_rank[b] * h->h_bm[b];
        voff64[b + 1] = voff64[b] + (int64_t)h->h_rank[b] * h->h_bn[b];
        toff[b + 1] = toff[b] + h->h_rank[b];
        h->n_rank_capped += hcap[b];
      }
      h->total_rank = toff[nblk];
      rc = upload(h->toff, toff, h->st);
      DevBuf<int64_t> du, dv;
      if (rc == HODLRDD_OK) rc = upload(du, uoff64, h->st);
      if (rc == HODLRDD_OK) rc = upload(dv, voff64, h->st);
      if (rc == HODLRDD_OK) rc = U64.alloc(std::max<int64_t>(uoff64[nblk], 1));
      if (rc == HODLRDD_OK) rc = V64.alloc(std::max<int64_t>(voff64[nblk], 1));
      if (rc == HODLRDD_OK) rc = h->piv_sigma.alloc(std::max<int64_t>(h->total_rank, 1));
      if (rc == HODLRDD_OK) rc = h->piv_tau.alloc(std::max<int64_t>(h->total_rank, 1));
      if (rc == HODLRDD_OK && cudaStreamSynchronize(h->st) != cudaSuccess) rc = HODLRDD_ERR_CUDA;
      // blocks whose factors are in the pool move to their place; the others
      // (the pool was full, or there is no pool) are recomputed below
      bool again = false;
      for (auto& B : bins) {
        std::vector<int32_t> rest;
        for (int32_t b : B.list)
          if (h->h_rank[b] > 0 && (!base.pool || hpoff[b] < 0)) rest.push_back(b);
        again |= !rest.empty();
        B.list.swap(rest);
        if (rc == HODLRDD_OK && !B.list.empty()) rc = upload(B.dlist, B.list, h->st);
      }
      if (rc == HODLRDD_OK && base.pool) {
        k_aca_compact<<<(int)std::min<int64_t>(nblk, (int64_t)dev_sms * 8), 256, 0, h->st>>>(
            nblk, poff.p, h->rank.p, h->bm.p, h->bn.p, pool.p, du.p, dv.p, h->toff.p, U64.p, V64.p,
            h->piv_sigma.p, h->piv_tau.p);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "ACA compaction", __FILE__, __LINE__);
        if (rc == HODLRDD_OK && cudaStreamSynchronize(h->st) != cudaSuccess) rc = HODLRDD_ERR_CUDA;
      }
      pool.release();
      DevBuf<int32_t> err;
      if (rc == HODLRDD_OK && again) rc = err.alloc(1);
      if (rc == HODLRDD_OK && again && cudaMemsetAsync(err.p, 0, sizeof(int32_t), h->st) != cudaSuccess)
        rc = HODLRDD_ERR_CUDA;
      if (rc == HODLRDD_OK && again && cudaStreamSynchronize(h->st) != cudaSuccess) rc = HODLRDD_ERR_CUDA;
      if (rc == HODLRDD_OK && again) {
        AcaArgs p2 = base;
        p2.pool = nullptr;
        p2.err = err.p;
        p2.U64 = U64.p;
        p2.V64 = V64.p;
        p2.uoff = du.p;
        p2.voff = dv.p;
        p2.toff = h->toff.p;
        p2.sig_out = h->piv_sigma.p;
        p2.tau_out = h->piv_tau.p;
        rc = launch_all(p2);  // the same arithmetic, factors written out
        int32_t herr = 0;
        if (rc == HODLRDD_OK && cudaMemcpy(&herr, err.p, sizeof herr, cudaMemcpyDeviceToHost) != cudaSuccess)
          rc = HODLRDD_ERR_CUDA;
        if (rc == HODLRDD_OK && herr) {
          set_error("ACA pass 2 did not reproduce pass 1");
          rc = HODLRDD_ERR_NUMERIC;
        }
      }
    }
  }
  for (auto& B : bins)
    if (B.st) cudaStreamDestroy(B.st);
  return rc;
}

}  // namespace hd
