// Factor packing (a6) and the HODLRdD matrix-vector product (a7 - a10).
//
// Algorithm 2 in GPU form, for a chunk of NR right-hand sides:
//   a7  gather    x_t[i] = x[perm[i]]                         (tree order)
//   a8  V-apply   t_b = V_b^T x_t(J_b) for every low-rank IL block b
//       U-apply   ylev[l](I) = sum_{b in IL(box)} U_b t_b, one owner warp per
//                 (level, target box, 64-row slice); IL blocks flagged dense at
//                 coarse levels are evaluated on the fly here
//   a9  near      per leaf box: sum over the near list (self and d' >= 1
//                 neighbours) and the leaf-level dense IL blocks, K(I,J) x_t(J)
//                 evaluated on the fly from the point coordinates, never stored
//   a10 combine   y[perm[i]] = sum_l ylev[l][i] + near(i)
// Every output row has exactly one writer per stage and a fixed summation
// order, so results are bitwise reproducible and no atomics touch y.
//
// Factor layout: block b's U_b (m x p) and V_b (n x p) are column-major with the
// row count padded to an even number (2-element vector loads), blocks in CSR
// order. 16-bit factors carry one FP32 scale per column (a power of two, so
// scaling is exact); the V-apply folds both scales of column k into t_b[k].
#include <algorithm>

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

template <class F> struct Fac;
template <> struct Fac<double> {
  using acc = double;
  static constexpr bool scaled = false;
  __device__ static double from(double v) { return v; }
  __host__ static double to_host(double v) { return v; }
  __device__ static void load2(const double* p, double& a, double& b) {
    double2 v = *reinterpret_cast<const double2*>(p);
    a = v.x; b = v.y;
  }
};
template <> struct Fac<float> {
  using acc = float;
  static constexpr bool scaled = false;
  __device__ static float from(double v) { return (float)v; }
  __host__ static double to_host(float v) { return v; }
  __device__ static void load2(const float* p, float& a, float& b) {
    float2 v = *reinterpret_cast<const float2*>(p);
    a = v.x; b = v.y;
  }
};
template <> struct Fac<__half> {
  using acc = float;
  static constexpr bool scaled = true;
  __device__ static __half from(double v) { return __float2half_rn((float)v); }
  __host__ static double to_host(__half v) { return (double)__half2float(v); }
  __device__ static void load2(const __half* p, float& a, float& b) {
    float2 v = __half22float2(*reinterpret_cast<const __half2*>(p));
    a = v.x; b = v.y;
  }
};
template <> struct Fac<__nv_bfloat16> {
  using acc = float;
  static constexpr bool scaled = true;
  __device__ static __nv_bfloat16 from(double v) { return __float2bfloat16_rn((float)v); }
  __host__ static double to_host(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
  __device__ static void load2(const __nv_bfloat16* p, float& a, float& b) {
    float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
    a = v.x; b = v.y;
  }
};

constexpr int kWarpsPerCta = 8;

// ---------------------------------------------------------------- packing ----
// One CTA per block, one warp per factor column. 16-bit: column scale = the
// smallest power of two >= max |entry| (exact rescaling), entries stored / scale.
template <class F>
__global__ void k_pack(int64_t nblk, const int32_t* __restrict__ rank, const int32_t* __restrict__ bm,
                       const int32_t* __restrict__ bn, const double* __restrict__ U64,
                       const double* __restrict__ V64, const int64_t* __restrict__ uoff64,
                       const int64_t* __restrict__ voff64, const int64_t* __restrict__ uoff,
                       const int64_t* __restrict__ voff, const int64_t* __restrict__ toff, F* __restrict__ U,
                       F* __restrict__ V, float* __restrict__ su, float* __restrict__ sv) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t b = blockIdx.x; b < nblk; b += gridDim.x) {
    const int p = rank[b];
    if (p == 0) continue;
    for (int side = 0; side < 2; ++side) {
      const int64_t rows = side == 0 ? bm[b] : bn[b];
      const int64_t ld = pad_rows(rows);
      const double* src = side == 0 ? U64 + uoff64[b] : V64 + voff64[b];
      F* dst = side == 0 ? U + uoff[b] : V + voff[b];
      float* sc = side == 0 ? su : sv;
      for (int k = w; k < p; k += nw) {
        const double* col = src + (int64_t)k * rows;
        double scale = 1.0;
        if (Fac<F>::scaled) {
          double mx = 0.0;
          for (int64_t i = lane; i < rows; i += 32) mx = fmax(mx, fabs(col[i]));
          for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
          int e = 0;
          if (mx > 0.0) {
            frexp(mx, &e);  // mx = f * 2^e with f in [0.5, 1)
          }
          scale = mx > 0.0 ? ldexp(1.0, e) : 1.0;
          if (lane == 0) sc[toff[b] + k] = (float)scale;
        }
        const double inv = 1.0 / scale;
        for (int64_t i = lane; i < ld; i += 32) dst[(int64_t)k * ld + i] = Fac<F>::from(i < rows ? col[i] * inv : 0.0);
      }
    }
  }
}

// ----------------------------------------------------------------- matvec ----
template <class Acc, class IO, int NR>
__global__ void k_gather(const IO* __restrict__ x, const int32_t* __restrict__ perm, int64_t N, int ldx, int c0,
                         Acc* __restrict__ xt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const IO* src = x + (int64_t)perm[i] * ldx + c0;
#pragma unroll
    for (int r = 0; r < NR; ++r) xt[i * NR + r] = (Acc)src[r];
  }
}

// Sum 32 per-lane partial values across the warp; lane l ends with the total of
// value index l (butterfly halving: 31 shuffles for 32 sums).
template <class Acc>
__device__ __forceinline__ Acc transpose_reduce(Acc (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      Acc send = upper ? v[i] : v[i + off];
      Acc keep = upper ? v[i + off] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return v[0];
}

// t_b[k] = sv_k su_k sum_j V_b[j, k] x_t[J0 + j]   for the columns of one item.
// Item = {block, k0, kc}: up to 32 columns; processed CW = 32 / NR at a time.
template <class F, int NR>
__global__ void __launch_bounds__(256) k_vapply(const int4* __restrict__ items, int64_t nitems,
                                                const F* __restrict__ V, const int64_t* __restrict__ voff,
                                                const int32_t* __restrict__ bJ0, const int32_t* __restrict__ bn,
                                                const int64_t* __restrict__ toff, const float* __restrict__ su,
                                                const float* __restrict__ sv,
                                                const typename Fac<F>::acc* __restrict__ xt,
                                                typename Fac<F>::acc* __restrict__ t) {
  using Acc = typename Fac<F>::acc;
  constexpr int CW = 32 / NR;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it = warp; it < nitems; it += nwarps) {
    const int4 item = items[it];
    const int b = item.x;
    const int J0 = bJ0[b], n = bn[b];
    const int64_t ld = pad_rows(n);
    const F* Vb = V + voff[b];
    for (int c0 = item.y; c0 < item.y + item.z; c0 += CW) {
      const int kc = min(CW, item.y + item.z - c0);
      Acc acc[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) acc[i] = Acc(0);
      for (int j = 2 * lane; j < n; j += 64) {
        Acc x0[NR], x1[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          x0[r] = xt[(int64_t)(J0 + j) * NR + r];
          x1[r] = (j + 1 < n) ? xt[(int64_t)(J0 + j + 1) * NR + r] : Acc(0);
        }
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          if (c < kc) {
            Acc a, bb;
            Fac<F>::load2(Vb + (int64_t)(c0 + c) * ld + j, a, bb);
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[c * NR + r] += a * x0[r] + bb * x1[r];
          }
        }
      }
      Acc tot = transpose_reduce(acc);
      const int c = lane / NR, r = lane % NR;
      if (c < kc) {
        const int64_t col = toff[b] + c0 + c;
        if (Fac<F>::scaled) tot *= (Acc)(sv[col] * su[col]);
        t[col * NR + r] = tot;
      }
    }
  }
}

// ylev[l](rows) = sum over the IL blocks of the target box (low-rank: U_b t_b;
// dense at coarse levels: K(I,J) x_t(J) on the fly). One warp per item, 2 rows
// per lane. Item = {blk_begin, blk_end, row_start, nrows}; ulevel = level.
template <class F, int NR, bool FP64EVAL>
__global__ void __launch_bounds__(256) k_uapply(const int4* __restrict__ items, const int32_t* __restrict__ ulevel,
                                                int64_t nitems, int kappa, const F* __restrict__ U,
                                                const int64_t* __restrict__ uoff, const int32_t* __restrict__ rank,
                                                const int32_t* __restrict__ dense, const int32_t* __restrict__ bI0,
                                                const int32_t* __restrict__ bm, const int32_t* __restrict__ bJ0,
                                                const int32_t* __restrict__ bn,
                                                const int64_t* __restrict__ toff, const typename Fac<F>::acc* __restrict__ t,
                                                const typename Fac<F>::acc* __restrict__ xt, const void* __restrict__ pts,
                                                int64_t N, int d, int kid, double kc_const, double kscale,
                                                typename Fac<F>::acc* __restrict__ ylev) {
  using Acc = typename Fac<F>::acc;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it = warp; it < nitems; it += nwarps) {
    const int4 item = items[it];
    const int l = ulevel[it];
    const int row0 = item.z + 2 * lane;
    const bool v0 = 2 * lane < item.w, v1 = 2 * lane + 1 < item.w;
    Acc acc0[NR], acc1[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) { acc0[r] = Acc(0); acc1[r] = Acc(0); }
    for (int b = item.x; b < item.y; ++b) {
      if (dense[b]) {
        if (l == kappa) continue;  // leaf-level dense blocks belong to the near stage
        // on-the-fly K(I,J) x_t(J) for this lane's two rows
        const int J0 = bJ0[b], n = bn[b];
        Acc s0[NR], s1[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) { s0[r] = Acc(0); s1[r] = Acc(0); }
        if (FP64EVAL) {
          const double* P = static_cast<const double*>(pts);
          double xa[kMaxDim], xb[kMaxDim];
          for (int c = 0; c < d; ++c) {
            xa[c] = v0 ? P[(int64_t)c * N + row0] : 0.0;
            xb[c] = v1 ? P[(int64_t)c * N + row0 + 1] : 0.0;
          }
          for (int j = J0; j < J0 + n; ++j) {
            double sa = 0.0, sb = 0.0;
            for (int c = 0; c < d; ++c) {
              double pj = P[(int64_t)c * N + j];
              double da = xa[c] - pj, db = xb[c] - pj;
              sa += da * da;
              sb += db * db;
            }
            double fa = f64fast_of_s(kid, sa, kc_const), fb = f64fast_of_s(kid, sb, kc_const);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
              Acc xv = xt[(int64_t)j * NR + r];
              s0[r] += (Acc)fa * xv;
              s1[r] += (Acc)fb * xv;
            }
          }
        } else {
          const float* P = static_cast<const float*>(pts);
          float xa[kMaxDim], xb[kMaxDim];
          for (int c = 0; c < d; ++c) {
            xa[c] = v0 ? P[(int64_t)c * N + row0] : 0.f;
            xb[c] = v1 ? P[(int64_t)c * N + row0 + 1] : 0.f;
          }
          const float kcf = (float)kc_const;
          for (int j = J0; j < J0 + n; ++j) {
            float sa = 0.f, sb = 0.f;
            for (int c = 0; c < d; ++c) {
              float pj = P[(int64_t)c * N + j];
              float da = xa[c] - pj, db = xb[c] - pj;
              sa += da * da;
              sb += db * db;
            }
            float fa = f32_of_s(kid, sa, kcf), fb = f32_of_s(kid, sb, kcf);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
              Acc xv = xt[(int64_t)j * NR + r];
              s0[r] += (Acc)fa * xv;
              s1[r] += (Acc)fb * xv;
            }
          }
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          acc0[r] += (Acc)kscale * s0[r];
          acc1[r] += (Acc)kscale * s1[r];
        }
        continue;
      }
      const int p = rank[b];
      if (p == 0) continue;
      const F* Ub = U + uoff[b];
      const int64_t ldU = pad_rows((int64_t)bm[b]);  // column stride: padded target-box height
      const int64_t rl = (int64_t)(row0 - bI0[b]);
      const Acc* tb = t + toff[b] * NR;
      if (v0) {
        for (int k = 0; k < p; ++k) {
          Acc a, bb;
          Fac<F>::load2(Ub + (int64_t)k * ldU + rl, a, bb);
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            Acc tv = tb[k * NR + r];
            acc0[r] += a * tv;
            acc1[r] += bb * tv;
          }
        }
      }
    }
    const int64_t yrow = (int64_t)(l - 1) * N + row0;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (v0) ylev[yrow * NR + r] = acc0[r];
      if (v1) ylev[(yrow + 1) * NR + r] = acc1[r];
    }
  }
}

// Near field and final combination for one leaf box per warp. Rows are handled
// G at a time with 32 / G source stripes; stripes are summed by shuffles.
template <class Acc, class IO, int NR, bool FP64EVAL>
__global__ void __launch_bounds__(256) k_near(const int4* __restrict__ items, int64_t nitems,
                                              const int32_t* __restrict__ near_src,
                                              const int32_t* __restrict__ leaf_start, const Acc* __restrict__ xt,
                                              const void* __restrict__ pts, int64_t N, int d, int kid,
                                              double kc_const, double kscale, double kdiag,
                                              const Acc* __restrict__ ylev, int kappa,
                                              const int32_t* __restrict__ perm, IO* __restrict__ y, int ldy, int c0) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it = warp; it < nitems; it += nwarps) {
    const int4 item = items[it];
    const int I0 = item.x, m = item.y;
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
      if (FP64EVAL) {
        const double* P = static_cast<const double*>(pts);
        double xr[kMaxDim];
        for (int c = 0; c < d; ++c) xr[c] = valid ? P[(int64_t)c * N + row] : 0.0;
        for (int e = item.z; e < item.w; ++e) {
          const int src = near_src[e];
          const int J0 = leaf_start[src], J1 = leaf_start[src + 1];
          for (int j = J0 + stripe; j < J1; j += S) {
            double s = 0.0;
            for (int c = 0; c < d; ++c) {
              double dd = xr[c] - P[(int64_t)c * N + j];
              s += dd * dd;
            }
            double f = f64fast_of_s(kid, s, kc_const);
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[r] += (Acc)f * xt[(int64_t)j * NR + r];
          }
        }
      } else {
        const float* P = static_cast<const float*>(pts);
        const float kcf = (float)kc_const;
        float xr[kMaxDim];
        for (int c = 0; c < d; ++c) xr[c] = valid ? P[(int64_t)c * N + row] : 0.f;
        for (int e = item.z; e < item.w; ++e) {
          const int src = near_src[e];
          const int J0 = leaf_start[src], J1 = leaf_start[src + 1];
          for (int j = J0 + stripe; j < J1; j += S) {
            float s = 0.f;
            for (int c = 0; c < d; ++c) {
              float dd = xr[c] - P[(int64_t)c * N + j];
              s += dd * dd;
            }
            float f = f32_of_s(kid, s, kcf);
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[r] += (Acc)f * xt[(int64_t)j * NR + r];
          }
        }
      }
#pragma unroll
      for (int r = 0; r < NR; ++r)
        for (int o = G; o < 32; o <<= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
      if (stripe == 0 && valid) {
        const int64_t orow = perm[row];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          Acc tot = (Acc)kscale * acc[r] + (Acc)kdiag * xt[(int64_t)row * NR + r];
          for (int l = 1; l <= kappa; ++l) tot += ylev[((int64_t)(l - 1) * N + row) * NR + r];
          y[orow * ldy + c0 + r] = (IO)tot;
        }
      }
    }
  }
}

int grid_warps(int64_t items, int dev_sms) {
  int64_t ctas = (items + kWarpsPerCta - 1) / kWarpsPerCta;
  int64_t cap = (int64_t)dev_sms * 8;
  if (ctas > cap) ctas = cap;
  if (ctas < 1) ctas = 1;
  return (int)ctas;
}

template <class F>
int pack_typed(hodlrdd_s* h, const DevBuf<double>& U64, const DevBuf<double>& V64, const DevBuf<int64_t>& du64,
               const DevBuf<int64_t>& dv64, const DevBuf<int64_t>& duoff, const DevBuf<int64_t>& dvoff,
               int64_t uelems, int64_t velems) {
  HD_TRY(h->U.alloc(std::max<int64_t>(uelems, 1) * sizeof(F)));
  HD_TRY(h->V.alloc(std::max<int64_t>(velems, 1) * sizeof(F)));
  if (Fac<F>::scaled) {
    HD_TRY(h->su.alloc(std::max<int64_t>(h->total_rank, 1)));
    HD_TRY(h->sv.alloc(std::max<int64_t>(h->total_rank, 1)));
  } else {
    h->su.release();
    h->sv.release();
  }
  if (h->nblk > 0) {
    int g = (int)std::min<int64_t>(h->nblk, 152 * 32);
    k_pack<F><<<g, 256, 0, h->st>>>(h->nblk, h->rank.p, h->bm.p, h->bn.p, U64.p, V64.p, du64.p, dv64.p, duoff.p,
                                    dvoff.p, h->toff.p, reinterpret_cast<F*>(h->U.p), reinterpret_cast<F*>(h->V.p),
                                    h->su.p, h->sv.p);
    HD_CUDA(cudaGetLastError());
  }
  HD_CUDA(cudaStreamSynchronize(h->st));
  return HODLRDD_OK;
}

}  // namespace

int pack_factors(hodlrdd_s* h, const DevBuf<double>& U64, const DevBuf<double>& V64,
                 const std::vector<int64_t>& uoff64, const std::vector<int64_t>& voff64) {
  const int64_t nblk = h->nblk;
  std::vector<int64_t> uoff(nblk + 1, 0), voff(nblk + 1, 0);
  h->factor_elems = 0;
  for (int64_t b = 0; b < nblk; ++b) {
    const int64_t p = h->h_rank[b];
    uoff[b + 1] = uoff[b] + p * pad_rows(h->h_bm[b]);
    voff[b + 1] = voff[b] + p * pad_rows(h->h_bn[b]);
    h->factor_elems += p * (h->h_bm[b] + h->h_bn[b]);
  }
  DevBuf<int64_t> du64, dv64;
  HD_TRY(upload(du64, uoff64, h->st));
  HD_TRY(upload(dv64, voff64, h->st));
  HD_TRY(upload(h->uoff, uoff, h->st));
  HD_TRY(upload(h->voff, voff, h->st));
  HD_CUDA(cudaStreamSynchronize(h->st));
  const int64_t ue = uoff[nblk], ve = voff[nblk];
  int rc;
  switch (h->opt.precision) {
    case HODLRDD_PREC_FP64: rc = pack_typed<double>(h, U64, V64, du64, dv64, h->uoff, h->voff, ue, ve); break;
    case HODLRDD_PREC_FP32: rc = pack_typed<float>(h, U64, V64, du64, dv64, h->uoff, h->voff, ue, ve); break;
    case HODLRDD_PREC_FP16: rc = pack_typed<__half>(h, U64, V64, du64, dv64, h->uoff, h->voff, ue, ve); break;
    default: rc = pack_typed<__nv_bfloat16>(h, U64, V64, du64, dv64, h->uoff, h->voff, ue, ve); break;
  }
  if (rc != HODLRDD_OK) return rc;
  h->factor_bytes = (ue + ve) * (int64_t)elem_size(h->opt.precision) +
                    (h->opt.precision >= HODLRDD_PREC_FP16 ? 2 * h->total_rank * 4 : 0);
  return HODLRDD_OK;
}

int build_plan(hodlrdd_s* h) {
  Plan& P = h->plan;
  const int64_t nblk = h->nblk;
  std::vector<int4> vitems;
  for (int64_t b = 0; b < nblk; ++b)
    for (int k0 = 0; k0 < h->h_rank[b]; k0 += 32)
      vitems.push_back(make_int4((int)b, k0, std::min(32, h->h_rank[b] - k0), 0));
  std::stable_sort(vitems.begin(), vitems.end(),
                   [&](const int4& a, const int4& c) { return h->h_bn[a.x] > h->h_bn[c.x]; });
  std::vector<int4> uitems;
  std::vector<int32_t> ulevel;
  for (int l = 1; l <= h->kappa; ++l) {
    const Level& L = h->lv[l];
    for (int64_t i = 0; i < L.nb; ++i) {
      const int32_t b0 = (int32_t)(h->h_blk_off[l] + L.h_iloff[i]);
      const int32_t b1 = (int32_t)(h->h_blk_off[l] + L.h_iloff[i + 1]);
      bool work = false;
      for (int32_t b = b0; b < b1 && !work; ++b)
        work = h->h_rank[b] > 0 || (h->h_dense[b] && l < h->kappa);
      if (!work) continue;
      const int32_t I0 = L.h_bstart[i], m = L.h_bstart[i + 1] - I0;
      for (int32_t r = 0; r < m; r += 64) {
        uitems.push_back(make_int4(b0, b1, I0 + r, std::min(64, m - r)));
        ulevel.push_back(l);
      }
    }
  }
  // near list per leaf box: self + d' >= 1 neighbours, then dense leaf-level IL blocks
  const Level& Lk = h->lv[h->kappa];
  std::vector<int4> nitems;
  std::vector<int32_t> near_src;
  h->dense_pairs = 0;
  for (int64_t i = 0; i < Lk.nb; ++i) {
    const int32_t I0 = Lk.h_bstart[i], m = Lk.h_bstart[i + 1] - I0;
    const int32_t e0 = (int32_t)near_src.size();
    for (int32_t e = h->h_nearoff[i]; e < h->h_nearoff[i + 1]; ++e) {
      int32_t j = h->h_nearidx[e];
      near_src.push_back(j);
      h->dense_pairs += (int64_t)m * (Lk.h_bstart[j + 1] - Lk.h_bstart[j]);
    }
    if (h->kappa >= 1) {
      const int64_t b0 = h->h_blk_off[h->kappa] + Lk.h_iloff[i], b1 = h->h_blk_off[h->kappa] + Lk.h_iloff[i + 1];
      for (int64_t b = b0; b < b1; ++b)
        if (h->h_dense[b]) {
          near_src.push_back(h->h_bsj[b]);
          h->dense_pairs += (int64_t)m * h->h_bn[b];
        }
    }
    nitems.push_back(make_int4(I0, m, e0, (int32_t)near_src.size()));
  }
  for (int64_t b = 0; b < nblk; ++b)
    if (h->h_dense[b] && h->h_blevel[b] < h->kappa) h->dense_pairs += (int64_t)h->h_bm[b] * h->h_bn[b];
  std::vector<int4> nsorted = nitems;
  cudaStream_t st = h->st;
  P.n_vitems = (int64_t)vitems.size();
  P.n_uitems = (int64_t)uitems.size();
  P.n_nitems = (int64_t)nsorted.size();
  P.n_near_src = (int64_t)near_src.size();
  HD_TRY(upload(P.vitems, vitems, st));
  HD_TRY(upload(P.uitems, uitems, st));
  HD_TRY(upload(P.ulevel, ulevel, st));
  HD_TRY(upload(P.nitems, nsorted, st));
  HD_TRY(upload(P.near_src, near_src, st));
  HD_CUDA(cudaStreamSynchronize(st));
  return HODLRDD_OK;
}

int alloc_workspace(hodlrdd_s* h) {
  const int nr = 8;
  const size_t acc = h->opt.precision == HODLRDD_PREC_FP64 ? 8 : 4;
  HD_TRY(h->xt.alloc((size_t)h->N * nr * acc));
  HD_TRY(h->tbuf.alloc((size_t)std::max<int64_t>(h->total_rank, 1) * nr * acc));
  HD_TRY(h->ylev.alloc((size_t)std::max(h->kappa, 1) * h->N * nr * acc));
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

template <class F, class IO, int NR>
int matvec_chunk(hodlrdd_s* h, const IO* x, IO* y, int ldx, int c0, cudaStream_t st) {
  using Acc = typename Fac<F>::acc;
  constexpr bool F64 = std::is_same<F, double>::value;
  const Plan& P = h->plan;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  Acc* xt = reinterpret_cast<Acc*>(h->xt.p);
  Acc* t = reinterpret_cast<Acc*>(h->tbuf.p);
  Acc* yl = reinterpret_cast<Acc*>(h->ylev.p);
  const void* pts = F64 ? (const void*)h->pts64.p : (const void*)h->pts32.p;
  const double kc = kernel_const(h->K);
  cudaEvent_t ev[5];
  const bool prof = h->profiling;
  if (prof) {
    HD_TRY(chunk_events(h, ev));
    HD_CUDA(cudaEventRecord(ev[0], st));
  }
  k_gather<Acc, IO, NR><<<(int)std::min<int64_t>((h->N + 255) / 256, sms * 16), 256, 0, st>>>(x, h->perm.p, h->N, ldx,
                                                                                              c0, xt);
  h->launches += 1;
  if (prof) HD_CUDA(cudaEventRecord(ev[1], st));
  if (h->kappa >= 1) {
    HD_CUDA(cudaMemsetAsync(yl, 0, (size_t)h->kappa * h->N * NR * sizeof(Acc), st));
    if (P.n_vitems > 0) {
      k_vapply<F, NR><<<grid_warps(P.n_vitems, sms), 32 * kWarpsPerCta, 0, st>>>(
          P.vitems.p, P.n_vitems, reinterpret_cast<const F*>(h->V.p), h->voff.p, h->bJ0.p, h->bn.p, h->toff.p,
          h->su.p, h->sv.p, xt, t);
      h->launches += 1;
    }
  }
  if (prof) HD_CUDA(cudaEventRecord(ev[2], st));
  if (h->kappa >= 1) {
    if (P.n_uitems > 0) {
      k_uapply<F, NR, F64><<<grid_warps(P.n_uitems, sms), 32 * kWarpsPerCta, 0, st>>>(
          P.uitems.p, P.ulevel.p, P.n_uitems, h->kappa, reinterpret_cast<const F*>(h->U.p), h->uoff.p, h->rank.p,
          h->dense.p, h->bI0.p, h->bm.p, h->bJ0.p, h->bn.p, h->toff.p, t, xt, pts, h->N, h->d, h->K.id, kc, h->K.scale, yl);
      h->launches += 1;
    }
  }
  if (prof) HD_CUDA(cudaEventRecord(ev[3], st));
  k_near<Acc, IO, NR, F64><<<grid_warps(P.n_nitems, sms), 32 * kWarpsPerCta, 0, st>>>(
      P.nitems.p, P.n_nitems, P.near_src.p, h->lv[h->kappa].bstart.p, xt, pts, h->N, h->d, h->K.id, kc, h->K.scale,
      h->K.diag, yl, h->kappa, h->perm.p, y, ldx, c0);
  h->launches += 1;
  HD_CUDA(cudaGetLastError());
  if (prof) HD_CUDA(cudaEventRecord(ev[4], st));
  return HODLRDD_OK;
}

template <class F, class IO>
int matvec_typed(hodlrdd_s* h, const IO* x, IO* y, int nrhs, cudaStream_t st) {
  int c0 = 0;
  while (c0 < nrhs) {
    const int rem = nrhs - c0;
    if (rem >= 8) { HD_TRY((matvec_chunk<F, IO, 8>(h, x, y, nrhs, c0, st))); c0 += 8; }
    else if (rem >= 4) { HD_TRY((matvec_chunk<F, IO, 4>(h, x, y, nrhs, c0, st))); c0 += 4; }
    else if (rem >= 2) { HD_TRY((matvec_chunk<F, IO, 2>(h, x, y, nrhs, c0, st))); c0 += 2; }
    else { HD_TRY((matvec_chunk<F, IO, 1>(h, x, y, nrhs, c0, st))); c0 += 1; }
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
template <class F>
int unpack_typed(hodlrdd_s* h, int64_t b, double* U, double* V) {
  const int p = h->h_rank[b];
  if (p == 0) return HODLRDD_OK;
  std::vector<int64_t> uo(2), vo(2), to(1);
  HD_CUDA(cudaMemcpy(uo.data(), h->uoff.p + b, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost));
  HD_CUDA(cudaMemcpy(vo.data(), h->voff.p + b, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost));
  HD_CUDA(cudaMemcpy(to.data(), h->toff.p + b, sizeof(int64_t), cudaMemcpyDeviceToHost));
  for (int side = 0; side < 2; ++side) {
    const int64_t rows = side == 0 ? h->h_bm[b] : h->h_bn[b];
    const int64_t ld = pad_rows(rows);
    std::vector<F> buf((size_t)ld * p);
    const F* src = reinterpret_cast<const F*>(side == 0 ? h->U.p : h->V.p) + (side == 0 ? uo[0] : vo[0]);
    HD_CUDA(cudaMemcpy(buf.data(), src, buf.size() * sizeof(F), cudaMemcpyDeviceToHost));
    std::vector<float> sc(p, 1.0f);
    if (Fac<F>::scaled)
      HD_CUDA(cudaMemcpy(sc.data(), (side == 0 ? h->su.p : h->sv.p) + to[0], p * sizeof(float),
                         cudaMemcpyDeviceToHost));
    double* out = side == 0 ? U : V;
    if (!out) continue;
    for (int k = 0; k < p; ++k)
      for (int64_t i = 0; i < rows; ++i) out[k * rows + i] = Fac<F>::to_host(buf[k * ld + i]) * (double)sc[k];
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

}  // namespace hd
