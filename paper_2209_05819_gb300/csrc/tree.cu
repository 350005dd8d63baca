// 2^d tree and interaction lists on the device.
//
//  a1  bounding hyper-cube and integer cell coordinates (Section "Construction of
//      the tree": a hyper-cube C holding the particles, split 2^d-ways per level);
//  a2  Morton keys and a stable sort -> tree order;
//  a3  per-level box tables; the leaf level kappa is the first level whose boxes
//      all hold at most leaf_size points (Algorithm 1's level rule);
//  a4  interaction lists IL = clan ∩ (vertex-sharing ∪ far-field) (Table
//      "Notations" and the HODLRdD admissibility condition) and the leaf near
//      lists (self and d' >= 1 neighbours, Algorithm 2's dense part).
//
// All integer work is deterministic: the outputs are bit-identical from run to
// run. Compiled with FP contraction off so the cell coordinates round exactly as
// (x - lo) * inv in plain FP64.
#include <cub/cub.cuh>

#include "internal.cuh"

namespace hd {
namespace {

constexpr int TPB = 256;

inline int grid_for(int64_t n, int tpb = TPB, int cap = 152 * 16) {
  int64_t g = (n + tpb - 1) / tpb;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

__global__ void k_minmax(const double* __restrict__ pts, int64_t N, int d, double* __restrict__ part) {
  // part per block: d minima, d maxima, then 1.0 if any coordinate was NaN / Inf.
  __shared__ double smn[TPB / 32], smx[TPB / 32];
  __shared__ int sbad;
  if (threadIdx.x == 0) sbad = 0;
  __syncthreads();
  int bad = 0;
  const size_t stride = 2 * (size_t)d + 1;
  for (int k = 0; k < d; ++k) {
    double mn = INFINITY, mx = -INFINITY;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
      double v = pts[i * d + k];
      if (!isfinite(v)) bad = 1;
      mn = fmin(mn, v);
      mx = fmax(mx, v);
    }
    for (int o = 16; o; o >>= 1) {
      mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
      smn[threadIdx.x >> 5] = mn;
      smx[threadIdx.x >> 5] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        mn = fmin(mn, smn[w]);
        mx = fmax(mx, smx[w]);
      }
      part[(size_t)blockIdx.x * stride + k] = mn;
      part[(size_t)blockIdx.x * stride + d + k] = mx;
    }
    __syncthreads();
  }
  if (bad) atomicOr(&sbad, 1);
  __syncthreads();
  if (threadIdx.x == 0) part[(size_t)blockIdx.x * stride + 2 * d] = sbad ? 1.0 : 0.0;
}

// cube = {lo[0..d), side, inv, finite-flag}
__global__ void k_cube(const double* __restrict__ part, int nparts, int d, int B, double* __restrict__ cube) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const size_t stride = 2 * (size_t)d + 1;
  double ext = 0.0;
  bool finite = true;
  for (int b = 0; b < nparts; ++b)
    if (part[(size_t)b * stride + 2 * d] != 0.0) finite = false;
  for (int k = 0; k < d; ++k) {
    double mn = part[k], mx = part[d + k];
    for (int b = 1; b < nparts; ++b) {
      mn = fmin(mn, part[(size_t)b * stride + k]);
      mx = fmax(mx, part[(size_t)b * stride + d + k]);
    }
    cube[k] = mn;
    ext = fmax(ext, mx - mn);
  }
  double side = ext > 0.0 ? ext * (1.0 + 0x1p-40) : 1.0;
  cube[d] = side;
  cube[d + 1] = ldexp(1.0, B) / side;
  cube[d + 2] = finite ? 1.0 : 0.0;
}

// Integer coordinate q_k = min(floor((x_k - lo_k) * inv), 2^B - 1); the key puts
// bit b of q_k at position d*b + k (level digits from coarse to fine).
__global__ void k_morton(const double* __restrict__ pts, int64_t N, int d, int B, const double* __restrict__ cube,
                         uint64_t* __restrict__ keys, int32_t* __restrict__ idx) {
  const double inv = cube[d + 1];
  const uint64_t maxc = (uint64_t(1) << B) - 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t key = 0;
    for (int k = 0; k < d; ++k) {
      double t = (pts[i * d + k] - cube[k]) * inv;
      double f = floor(t);
      if (f < 0.0) f = 0.0;
      uint64_t q = (uint64_t)f;
      if (q > maxc) q = maxc;
      for (int b = 0; b < B; ++b) key |= ((q >> b) & 1u) << (d * b + k);
    }
    keys[i] = key;
    idx[i] = (int32_t)i;
  }
}

__global__ void k_gather_points(const double* __restrict__ pts, const int32_t* __restrict__ perm, int64_t N, int d,
                                double* __restrict__ p64, float* __restrict__ p32) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t o = perm[i];
    for (int k = 0; k < d; ++k) {
      double v = pts[o * d + k];
      p64[(size_t)k * N + i] = v;
      p32[(size_t)k * N + i] = (float)v;
    }
  }
}

// dl[i] (i >= 1): the coarsest level at which point i starts a new box.
__global__ void k_first_level(const uint64_t* __restrict__ skey, int64_t N, int d, int B, int8_t* __restrict__ dl) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    if (i == 0) {
      dl[0] = 0;
      continue;
    }
    uint64_t x = skey[i] ^ skey[i - 1];
    if (x == 0) {
      dl[i] = 127;
    } else {
      int t = 63 - __clzll((long long)x);
      dl[i] = (int8_t)(B - t / d);
    }
  }
}

__global__ void k_flags(const int8_t* __restrict__ dl, int64_t N, int l, int32_t* __restrict__ flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || dl[i] <= l) ? 1 : 0;
}

// incl = inclusive scan of flags; box id = incl - 1 (written in place).
__global__ void k_box_starts(const int32_t* __restrict__ flag, int32_t* __restrict__ bid, int64_t N,
                             int32_t* __restrict__ bstart) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t b = bid[i] - 1;
    bid[i] = b;
    if (flag[i]) bstart[b] = (int32_t)i;
    if (i == N - 1) bstart[b + 1] = (int32_t)N;
  }
}

__global__ void k_box_keys(const int32_t* __restrict__ bstart, int64_t nb, const uint64_t* __restrict__ skey,
                           int shift, uint64_t* __restrict__ bkey, int32_t* __restrict__ maxocc) {
  int32_t local = 0;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
    bkey[b] = skey[bstart[b]] >> shift;
    local = max(local, bstart[b + 1] - bstart[b]);
  }
  for (int o = 16; o; o >>= 1) local = max(local, __shfl_xor_sync(0xffffffffu, local, o));
  if ((threadIdx.x & 31) == 0) atomicMax(maxocc, local);
}

// cfirst[P] = box id at the child level of the first point of parent box P.
__global__ void k_children(const int32_t* __restrict__ bstart, int64_t nb, const int32_t* __restrict__ bid_child,
                           int64_t nb_child, int32_t* __restrict__ cfirst) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b <= nb; b += (int64_t)gridDim.x * blockDim.x)
    cfirst[b] = b < nb ? bid_child[bstart[b]] : (int32_t)nb_child;
}

__device__ __forceinline__ uint64_t enc(const int64_t* c, int d, int bits) {
  uint64_t key = 0;
  for (int b = 0; b < bits; ++b)
    for (int k = 0; k < d; ++k) key |= (uint64_t)((c[k] >> b) & 1) << (d * b + k);
  return key;
}

__device__ __forceinline__ void dec(uint64_t key, int d, int bits, int64_t* c) {
  for (int k = 0; k < d; ++k) c[k] = 0;
  for (int b = 0; b < bits; ++b)
    for (int k = 0; k < d; ++k) c[k] |= (int64_t)((key >> (d * b + k)) & 1u) << b;
}

__device__ __forceinline__ int64_t find_box(const uint64_t* __restrict__ a, int64_t n, uint64_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return (lo < n && a[lo] == key) ? lo : -1;
}

// Interaction list of every box at level l >= 1. Candidates are the children of
// the parent and of each parent-level box sharing a face of dimension > amax
// with the parent (offset in {-1,0,1}^d with more than amax zeros; amax = 0 for
// HODLRdD, i.e. a d' >= 1 hyper-surface); a candidate j != i is kept when far
// (Chebyshev index distance >= 2) or touching along a face of dimension <= amax
// (for HODLRdD: vertex-sharing, all |delta| = 1).
template <bool FILL>
__global__ void k_il(int d, int l, int amax, int64_t nb, const uint64_t* __restrict__ bkey, int64_t nbp,
                     const uint64_t* __restrict__ pkey, const int32_t* __restrict__ pcfirst,
                     const int32_t* __restrict__ off, int32_t* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  int64_t c[kMaxDim], p[kMaxDim], q[kMaxDim], cj[kMaxDim];
  dec(bkey[i], d, l, c);
  for (int k = 0; k < d; ++k) p[k] = c[k] >> 1;
  const int64_t sidep = (int64_t)1 << (l - 1);
  int nd = 1;
  for (int k = 0; k < d; ++k) nd *= 3;
  int32_t cnt = 0;
  int64_t pos = FILL ? off[i] : 0;
  for (int t = 0; t < nd; ++t) {
    int tt = t;
    int zeros = 0;
    bool ok = true;
    for (int k = 0; k < d; ++k) {
      int dk = tt % 3 - 1;
      tt /= 3;
      q[k] = p[k] + dk;
      if (dk == 0) ++zeros;
      if (q[k] < 0 || q[k] >= sidep) ok = false;
    }
    if (!ok || zeros <= amax) continue;  // the parent itself has d zeros
    int64_t P = find_box(pkey, nbp, enc(q, d, l - 1));
    if (P < 0) continue;
    for (int32_t j = pcfirst[P]; j < pcfirst[P + 1]; ++j) {
      if (j == i) continue;
      dec(bkey[j], d, l, cj);
      int64_t cheb = 0;
      int jz = 0;
      for (int k = 0; k < d; ++k) {
        int64_t a = llabs(cj[k] - c[k]);
        cheb = max(cheb, a);
        if (a == 0) ++jz;
      }
      if (cheb >= 2 || jz <= amax) {
        if (FILL) out[pos++] = j; else ++cnt;
      }
    }
  }
  if (!FILL) out[i] = cnt;
}

// Leaf near list: the box itself and every leaf sharing a face of dimension >
// amax (HODLRdD: a d' >= 1 hyper-surface).
template <bool FILL>
__global__ void k_near(int d, int l, int amax, int64_t nb, const uint64_t* __restrict__ bkey,
                       const int32_t* __restrict__ off, int32_t* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  int64_t c[kMaxDim], q[kMaxDim];
  dec(bkey[i], d, l, c);
  const int64_t side = (int64_t)1 << l;
  int nd = 1;
  for (int k = 0; k < d; ++k) nd *= 3;
  int32_t cnt = 0;
  int64_t pos = FILL ? off[i] : 0;
  for (int t = 0; t < nd; ++t) {
    int tt = t;
    int zeros = 0;
    bool ok = true;
    for (int k = 0; k < d; ++k) {
      int dk = tt % 3 - 1;
      tt /= 3;
      q[k] = c[k] + dk;
      if (dk == 0) ++zeros;
      if (q[k] < 0 || q[k] >= side) ok = false;
    }
    if (!ok || zeros <= amax) continue;  // the box itself has d zeros
    int64_t j = find_box(bkey, nb, enc(q, d, l));
    if (j < 0) continue;
    if (FILL) out[pos++] = (int32_t)j; else ++cnt;
  }
  if (!FILL) out[i] = cnt;
}

__global__ void k_seg_keys(const int32_t* __restrict__ off, int64_t nb, const int32_t* __restrict__ idx,
                           uint64_t* __restrict__ keys) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x)
    for (int32_t e = off[i]; e < off[i + 1]; ++e) keys[e] = ((uint64_t)i << 32) | (uint32_t)idx[e];
}

__global__ void k_seg_unkey(const uint64_t* __restrict__ keys, int64_t n, int32_t* __restrict__ idx) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    idx[e] = (int32_t)(keys[e] & 0xffffffffu);
}

int inclusive_scan(const int32_t* in, int32_t* out, int64_t n, cudaStream_t st) {
  size_t bytes = 0;
  HD_CUDA(cub::DeviceScan::InclusiveSum(nullptr, bytes, in, out, (int)n, st));
  DevBuf<char> tmp;
  HD_TRY(tmp.alloc(bytes + 16));
  HD_CUDA(cub::DeviceScan::InclusiveSum(tmp.p, bytes, in, out, (int)n, st));
  HD_CUDA(cudaStreamSynchronize(st));
  return HODLRDD_OK;
}

// counts[nb] -> off[nb + 1] (exclusive), returns off[nb].
int counts_to_offsets(const int32_t* counts, int64_t nb, DevBuf<int32_t>& off, int64_t* total, cudaStream_t st) {
  HD_TRY(off.alloc(nb + 1));
  HD_CUDA(cudaMemsetAsync(off.p, 0, sizeof(int32_t), st));
  if (nb > 0) HD_TRY(inclusive_scan(counts, off.p + 1, nb, st));
  int32_t t = 0;
  HD_CUDA(cudaMemcpyAsync(&t, off.p + nb, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  HD_CUDA(cudaStreamSynchronize(st));
  *total = t;
  return HODLRDD_OK;
}

// Sort every CSR segment ascending (keys (segment << 32 | value), one global sort).
int sort_segments(const DevBuf<int32_t>& off, int64_t nb, DevBuf<int32_t>& idx, int64_t nnz, cudaStream_t st) {
  if (nnz == 0) return HODLRDD_OK;
  DevBuf<uint64_t> k0, k1;
  HD_TRY(k0.alloc(nnz));
  HD_TRY(k1.alloc(nnz));
  k_seg_keys<<<grid_for(nb), TPB, 0, st>>>(off.p, nb, idx.p, k0.p);
  int hi_bits = 1;
  while (((int64_t)1 << hi_bits) <= nb) ++hi_bits;
  size_t bytes = 0;
  HD_CUDA(cub::DeviceRadixSort::SortKeys(nullptr, bytes, k0.p, k1.p, (int)nnz, 0, 32 + hi_bits, st));
  DevBuf<char> tmp;
  HD_TRY(tmp.alloc(bytes + 16));
  HD_CUDA(cub::DeviceRadixSort::SortKeys(tmp.p, bytes, k0.p, k1.p, (int)nnz, 0, 32 + hi_bits, st));
  k_seg_unkey<<<grid_for(nnz), TPB, 0, st>>>(k1.p, nnz, idx.p);
  HD_CUDA(cudaGetLastError());
  HD_CUDA(cudaStreamSynchronize(st));
  return HODLRDD_OK;
}

}  // namespace

int build_tree(hodlrdd_s* h, const double* dpts) {
  cudaStream_t st = h->st;
  const int d = h->d;
  const int64_t N = h->N;
  h->B = (63 / d) < 32 ? 63 / d : 32;
  const int B = h->B;

  // a1: bounding cube
  const int g = grid_for(N);
  DevBuf<double> part, cube;
  HD_TRY(part.alloc((size_t)g * (2 * d + 1)));
  HD_TRY(cube.alloc(d + 3));
  k_minmax<<<g, TPB, 0, st>>>(dpts, N, d, part.p);
  k_cube<<<1, 32, 0, st>>>(part.p, g, d, B, cube.p);
  HD_CUDA(cudaGetLastError());
  std::vector<double> hc;
  HD_TRY(download(hc, cube.p, d + 3, st));
  HD_CUDA(cudaStreamSynchronize(st));
  if (hc[d + 2] != 1.0) {
    set_error("hodlrdd_build: points contain NaN or Inf");
    return HODLRDD_ERR_INVALID;
  }
  for (int k = 0; k < d; ++k) h->lo[k] = hc[k];
  h->side = hc[d];
  h->inv = hc[d + 1];

  // a2: keys and stable sort
  DevBuf<uint64_t> keys;
  DevBuf<int32_t> idx;
  HD_TRY(keys.alloc(N));
  HD_TRY(idx.alloc(N));
  HD_TRY(h->skey.alloc(N));
  HD_TRY(h->perm.alloc(N));
  k_morton<<<grid_for(N), TPB, 0, st>>>(dpts, N, d, B, cube.p, keys.p, idx.p);
  HD_CUDA(cudaGetLastError());
  {
    size_t bytes = 0;
    HD_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, bytes, keys.p, h->skey.p, idx.p, h->perm.p, (int)N, 0, d * B,
                                            st));
    DevBuf<char> tmp;
    HD_TRY(tmp.alloc(bytes + 16));
    HD_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, bytes, keys.p, h->skey.p, idx.p, h->perm.p, (int)N, 0, d * B,
                                            st));
    HD_CUDA(cudaStreamSynchronize(st));
  }
  keys.release();
  idx.release();
  HD_TRY(h->pts64.alloc((size_t)N * d));
  HD_TRY(h->pts32.alloc((size_t)N * d));
  k_gather_points<<<grid_for(N), TPB, 0, st>>>(dpts, h->perm.p, N, d, h->pts64.p, h->pts32.p);
  HD_CUDA(cudaGetLastError());

  // a3: level tables until every box holds at most leaf points (or l = B)
  DevBuf<int8_t> dl;
  DevBuf<int32_t> flag;
  DevBuf<int32_t> maxocc;
  HD_TRY(dl.alloc(N));
  HD_TRY(flag.alloc(N));
  HD_TRY(maxocc.alloc(1));
  k_first_level<<<grid_for(N), TPB, 0, st>>>(h->skey.p, N, d, B, dl.p);
  HD_CUDA(cudaGetLastError());
  h->lv.clear();
  for (int l = 0;; ++l) {
    h->lv.emplace_back();
    Level& L = h->lv.back();
    HD_TRY(L.bid.alloc(N));
    k_flags<<<grid_for(N), TPB, 0, st>>>(dl.p, N, l, flag.p);
    HD_CUDA(cudaGetLastError());
    HD_TRY(inclusive_scan(flag.p, L.bid.p, N, st));
    int32_t nb = 0;
    HD_CUDA(cudaMemcpyAsync(&nb, L.bid.p + N - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    HD_CUDA(cudaStreamSynchronize(st));
    L.nb = nb;
    HD_TRY(L.bstart.alloc(nb + 1));
    HD_TRY(L.bkey.alloc(nb));
    k_box_starts<<<grid_for(N), TPB, 0, st>>>(flag.p, L.bid.p, N, L.bstart.p);
    HD_CUDA(cudaMemsetAsync(maxocc.p, 0, sizeof(int32_t), st));
    k_box_keys<<<grid_for(nb), TPB, 0, st>>>(L.bstart.p, nb, h->skey.p, d * (B - l), L.bkey.p, maxocc.p);
    HD_CUDA(cudaGetLastError());
    int32_t mo = 0;
    HD_CUDA(cudaMemcpyAsync(&mo, maxocc.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    HD_TRY(download(L.h_bstart, L.bstart.p, nb + 1, st));
    HD_TRY(download(L.h_bkey, L.bkey.p, nb, st));
    HD_CUDA(cudaStreamSynchronize(st));
    if (mo <= h->leaf || l == B) {
      h->kappa = l;
      break;
    }
  }
  for (int l = 0; l < h->kappa; ++l) {
    Level& L = h->lv[l];
    HD_TRY(L.cfirst.alloc(L.nb + 1));
    k_children<<<grid_for(L.nb + 1), TPB, 0, st>>>(L.bstart.p, L.nb, h->lv[l + 1].bid.p, h->lv[l + 1].nb, L.cfirst.p);
    HD_CUDA(cudaGetLastError());
  }
  HD_TRY(download(h->h_perm, h->perm.p, N, st));
  HD_TRY(download(h->h_skey, h->skey.p, N, st));
  HD_CUDA(cudaStreamSynchronize(st));
  for (auto& L : h->lv) L.bid.release();
  return HODLRDD_OK;
}

int build_lists(hodlrdd_s* h) {
  cudaStream_t st = h->st;
  const int d = h->d;
  for (int l = 1; l <= h->kappa; ++l) {
    Level& L = h->lv[l];
    Level& P = h->lv[l - 1];
    DevBuf<int32_t> cnt;
    HD_TRY(cnt.alloc(L.nb));
    const int gb = (int)((L.nb + 127) / 128);
    k_il<false><<<gb, 128, 0, st>>>(d, l, h->opt.admissible_face_dim, L.nb, L.bkey.p, P.nb, P.bkey.p, P.cfirst.p, nullptr, cnt.p);
    HD_CUDA(cudaGetLastError());
    int64_t nnz = 0;
    HD_TRY(counts_to_offsets(cnt.p, L.nb, L.iloff, &nnz, st));
    if (nnz >= ((int64_t)1 << 31)) {
      set_error("interaction list too long for 32-bit offsets");
      return HODLRDD_ERR_UNSUPPORTED;
    }
    HD_TRY(L.ilidx.alloc(nnz));
    if (nnz) {
      k_il<true><<<gb, 128, 0, st>>>(d, l, h->opt.admissible_face_dim, L.nb, L.bkey.p, P.nb, P.bkey.p, P.cfirst.p, L.iloff.p, L.ilidx.p);
      HD_CUDA(cudaGetLastError());
      HD_TRY(sort_segments(L.iloff, L.nb, L.ilidx, nnz, st));
    }
    HD_TRY(download(L.h_iloff, L.iloff.p, L.nb + 1, st));
    HD_TRY(download(L.h_ilidx, L.ilidx.p, nnz, st));
    HD_CUDA(cudaStreamSynchronize(st));
  }
  Level& L = h->lv[h->kappa];
  DevBuf<int32_t> cnt;
  HD_TRY(cnt.alloc(L.nb));
  const int gb = (int)((L.nb + 127) / 128);
  k_near<false><<<gb, 128, 0, st>>>(d, h->kappa, h->opt.admissible_face_dim, L.nb, L.bkey.p, nullptr, cnt.p);
  HD_CUDA(cudaGetLastError());
  int64_t nnz = 0;
  HD_TRY(counts_to_offsets(cnt.p, L.nb, h->nearoff, &nnz, st));
  HD_TRY(h->nearidx.alloc(nnz));
  k_near<true><<<gb, 128, 0, st>>>(d, h->kappa, h->opt.admissible_face_dim, L.nb, L.bkey.p, h->nearoff.p, h->nearidx.p);
  HD_CUDA(cudaGetLastError());
  HD_TRY(sort_segments(h->nearoff, L.nb, h->nearidx, nnz, st));
  HD_TRY(download(h->h_nearoff, h->nearoff.p, L.nb + 1, st));
  HD_TRY(download(h->h_nearidx, h->nearidx.p, nnz, st));
  HD_CUDA(cudaStreamSynchronize(st));
  return HODLRDD_OK;
}

// Block table in CSR order (levels ascending, target box, source box).
int build_blocks(hodlrdd_s* h) {
  h->h_blk_off.assign(h->kappa + 2, 0);
  int64_t nblk = 0;
  for (int l = 1; l <= h->kappa; ++l) {
    h->h_blk_off[l] = nblk;
    nblk += (int64_t)h->lv[l].h_ilidx.size();
  }
  h->h_blk_off[0] = 0;
  h->h_blk_off[h->kappa + 1] = nblk;
  h->nblk = nblk;
  auto resize = [&](std::vector<int32_t>& v) { v.assign(nblk, 0); };
  resize(h->h_blevel); resize(h->h_bti); resize(h->h_bsj); resize(h->h_bI0); resize(h->h_bm);
  resize(h->h_bJ0); resize(h->h_bn);
  int64_t b = 0;
  for (int l = 1; l <= h->kappa; ++l) {
    const Level& L = h->lv[l];
    for (int64_t i = 0; i < L.nb; ++i)
      for (int32_t e = L.h_iloff[i]; e < L.h_iloff[i + 1]; ++e, ++b) {
        int32_t j = L.h_ilidx[e];
        h->h_blevel[b] = l;
        h->h_bti[b] = (int32_t)i;
        h->h_bsj[b] = j;
        h->h_bI0[b] = L.h_bstart[i];
        h->h_bm[b] = L.h_bstart[i + 1] - L.h_bstart[i];
        h->h_bJ0[b] = L.h_bstart[j];
        h->h_bn[b] = L.h_bstart[j + 1] - L.h_bstart[j];
      }
  }
  cudaStream_t st = h->st;
  HD_TRY(upload(h->bI0, h->h_bI0, st));
  HD_TRY(upload(h->bm, h->h_bm, st));
  HD_TRY(upload(h->bJ0, h->h_bJ0, st));
  HD_TRY(upload(h->bn, h->h_bn, st));
  HD_CUDA(cudaStreamSynchronize(st));
  return HODLRDD_OK;
}

}  // namespace hd
