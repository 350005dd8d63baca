// The memory-efficient apply of the low-rank blocks (Eq. keq2 and the remark
// after it: keep the pivots and the LU factors of K(sigma, tau), evaluate the
// rest of the kernel on the fly). For an IL block b = (I, J) of rank p whose
// partial-pivoted ACA picked rows sigma and columns tau,
//
//   K(I, J) x(J) ~ K(I, tau) U^-1 L^-1 K(sigma, J) x(J),   K(sigma, tau) = L U,
//
// with L(l, q) = u_q(sigma_l) lower triangular and U(q, l) = v_q(tau_l) unit
// upper triangular. A product runs in three steps:
//   rows:   s_b = K(sigma_b, J_b) x(J_b)        p |J| kernel evaluations
//   solve:  w_b = U_b^-1 (L_b^-1 s_b)           FP64: forward, then backward substitution;
//                                                FP32 form: w_b = W_b s_b with W_b = U_b^-1 L_b^-1
//                                                formed at the build (FP64)
//   cols:   y_l(I) += sum_b K(I, tau_b) w_b     p |I| kernel evaluations
// The handle keeps p^2 FP64 numbers per block instead of p (|I| + |J|) factor
// entries. The FP32 form evaluates the kernel on box-relative hi + lo
// coordinates (as the packed near field does); the FP64 form on the tree-order
// FP64 coordinates.
//
// Precision of the FP32 form. A trailing ACA term whose pivot L(q, q) is tiny
// against the leading pivots enters through s_q / L(q, q): the FP32 rounding of
// s_q (about eps |s|) grows by 1 / |L(q, q)|, and only the exact cancellation
// inside K(I, tau) U^-1 (the tiny column u_q) brings it back down, which FP32
// entries of K(I, tau) (again about eps) cannot reproduce. The cross term is
// about eps^2 |s| / |L(q, q)|. The FP32 form therefore keeps the leading terms
// while |L(q, q)| >= 2^-23 max_{m <= q} |L(m, m)| (FP32 unit roundoff): the
// dropped terms lie below what an FP32 evaluation of the block resolves and the
// cross term stays at about eps. The LU factors of the kept leading pivots are
// the leading blocks of L and U. The FP64 form keeps every term.
#include <algorithm>

#include "internal.cuh"
#include "pairs.cuh"

namespace hd {
namespace {

constexpr int kSkThreads = 256;  // threads of a row / column task
constexpr int kSkRows = 128;     // targets per task (two per thread over 64 .. 128 threads)
constexpr int kSkCap32 = 1024;   // staged sources per chunk, FP32 form
constexpr int kSkCap64 = 512;    // staged sources per chunk, FP64 form
constexpr int kSkMaxP = 1024;    // largest rank the triangular solves take (aca_max_rank <= this)
constexpr int kSkSolveWarps = 4; // warps per CTA of the solve (one block per warp)
constexpr double kSkTheta32 = 1.0 / 8388608.0;  // 2^-23: relative pivot kept by the FP32 form

// Threads per stripe: the smallest power of two holding nr targets two per thread.
__device__ __forceinline__ int stripe_width(int nr) {
  int G = 1;
  while (2 * G < nr) G <<= 1;
  return G;
}

// ---------------------------------------------------------------- FP32 form --

// Pivot rows against a source chunk: s[slot] (or a partial) = sum_j K(x_sigma, x_j) x_j
// for up to kSkRows rows of one source box. Targets are moved into the source
// box's frame by -(c_J - c_I) h_l with an error-free sum.
template <int D, int KID>
__global__ void __launch_bounds__(kSkThreads, 3)
    k_skel_rows(const SkTask* __restrict__ tasks, int64_t ntask, const int4* __restrict__ rows,
                const float4* __restrict__ boff, const float4* const* __restrict__ HiL,
                const float4* const* __restrict__ LoL, const float* __restrict__ xt, float kc, float kscale,
                float* __restrict__ s, float* __restrict__ part) {
  __shared__ float4 shi[kSkCap32];  // source hi (x_j in .w for D <= 3)
  __shared__ float4 slo[kSkCap32];
  __shared__ float sw[D > 3 ? kSkCap32 : 1];
  __shared__ float red[kSkThreads], red2[kSkThreads];
  const int tid = threadIdx.x;
  for (int64_t it = blockIdx.x; it < ntask; it += gridDim.x) {
    const SkTask T = tasks[it];
    const int nr = T.r1 - T.r0;
    const int G = stripe_width(nr);
    const int S = kSkThreads / G;
    const int gi = tid % G, stripe = tid / G;
    const bool va = gi < nr, vb = gi + G < nr;
    const float4* __restrict__ Hi = HiL[T.level];
    const float4* __restrict__ Lo = LoL[T.level];
    float4 tha = make_float4(0.f, 0.f, 0.f, 0.f), tla = tha, thb = tha, tlb = tha;
    auto load_target = [&](int r, float4& th, float4& tl) {
      const int4 R = rows[r];
      const float4 h = Hi[R.x], l = Lo[R.x], o = boff[R.z];
      float ex, ey, ez, ew;
      th = make_float4(two_sum(h.x, -o.x, ex), two_sum(h.y, -o.y, ey), two_sum(h.z, -o.z, ez),
                       two_sum(h.w, -o.w, ew));
      tl = make_float4(l.x + ex, l.y + ey, l.z + ez, l.w + ew);
    };
    if (va) load_target(T.r0 + gi, tha, tla);
    if (vb) load_target(T.r0 + gi + G, thb, tlb);
    __syncthreads();  // the previous task has finished with the staging arrays
    for (int k = tid; k < T.n; k += kSkThreads) {
      const int j = T.a0 + k;
      float4 h = Hi[j];
      if constexpr (D <= 3) h.w = xt[j];
      else sw[k] = xt[j];
      shi[k] = h;
      slo[k] = Lo[j];
    }
    __syncthreads();
    // compensated sums: the rounding of s reaches y through the interpolation
    // operator K(I, tau) K(sigma, tau)^-1, whose entries exceed one
    float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f, ca0 = 0.f, ca1 = 0.f, cb0 = 0.f, cb1 = 0.f;
    auto kadd = [](float& sum, float& comp, float term) {
      const float yv = term - comp;
      const float tv = sum + yv;
      comp = (tv - sum) - yv;
      sum = tv;
    };
    const int n = T.n;
    int f = stripe;
    for (; f + S < n; f += 2 * S) {
      const float4 h0 = shi[f], l0 = slo[f], h1 = shi[f + S], l1 = slo[f + S];
      const float w0 = D <= 3 ? h0.w : sw[f], w1 = D <= 3 ? h1.w : sw[f + S];
      kadd(a0, ca0, f32k_rn<KID>(sqdist2<D>(tha, tla, h0, l0), kc) * w0);
      kadd(b0, cb0, f32k_rn<KID>(sqdist2<D>(thb, tlb, h0, l0), kc) * w0);
      kadd(a1, ca1, f32k_rn<KID>(sqdist2<D>(tha, tla, h1, l1), kc) * w1);
      kadd(b1, cb1, f32k_rn<KID>(sqdist2<D>(thb, tlb, h1, l1), kc) * w1);
    }
    if (f < n) {
      const float4 h0 = shi[f], l0 = slo[f];
      const float w0 = D <= 3 ? h0.w : sw[f];
      kadd(a0, ca0, f32k_rn<KID>(sqdist2<D>(tha, tla, h0, l0), kc) * w0);
      kadd(b0, cb0, f32k_rn<KID>(sqdist2<D>(thb, tlb, h0, l0), kc) * w0);
    }
    red[tid] = (a0 - ca0) + (a1 - ca1);
    red2[tid] = (b0 - cb0) + (b1 - cb1);
    __syncthreads();
    if (stripe == 0) {
      float acc_a = 0.f, acc_b = 0.f, ca = 0.f, cb = 0.f;
      for (int q = 0; q < S; ++q) {
        kadd(acc_a, ca, red[q * G + gi]);
        kadd(acc_b, cb, red2[q * G + gi]);
      }
      acc_a -= ca;
      acc_b -= cb;
      if (T.pout < 0) {
        if (va) s[rows[T.r0 + gi].y] = kscale * acc_a;
        if (vb) s[rows[T.r0 + gi + G].y] = kscale * acc_b;
      } else {
        if (va) part[T.pout + gi] = acc_a;
        if (vb) part[T.pout + gi + G] = acc_b;
      }
    }
  }
}

// Targets of one box at one level against the pivot columns of all its
// low-rank IL blocks: ylev[(l - 1) N + i] = scale * sum_q K(x_i, x_tau_q) w_q.
// Columns are moved into the target box's frame by (c_J - c_I) h_l.
template <int D, int KID>
__global__ void __launch_bounds__(kSkThreads, 3)
    k_skel_cols(const SkTask* __restrict__ tasks, int64_t ntask, const int2* __restrict__ cols,
                const float4* __restrict__ boff, const float4* const* __restrict__ HiL,
                const float4* const* __restrict__ LoL, const float* __restrict__ w, float kc, float kscale,
                float* __restrict__ ylev, int64_t N) {
  __shared__ float4 shi[kSkCap32];
  __shared__ float4 slo[kSkCap32];
  __shared__ float sw[D > 3 ? kSkCap32 : 1];
  __shared__ float red[kSkThreads], red2[kSkThreads];
  const int tid = threadIdx.x;
  for (int64_t it = blockIdx.x; it < ntask; it += gridDim.x) {
    const SkTask T = tasks[it];
    const int nr = T.n;
    const int G = stripe_width(nr);
    const int S = kSkThreads / G;
    const int gi = tid % G, stripe = tid / G;
    const bool va = gi < nr, vb = gi + G < nr;
    const float4* __restrict__ Hi = HiL[T.level];
    const float4* __restrict__ Lo = LoL[T.level];
    float4 tha = make_float4(0.f, 0.f, 0.f, 0.f), tla = tha, thb = tha, tlb = tha;
    if (va) {
      tha = Hi[T.a0 + gi];
      tla = Lo[T.a0 + gi];
    }
    if (vb) {
      thb = Hi[T.a0 + gi + G];
      tlb = Lo[T.a0 + gi + G];
    }
    float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
    for (int c = T.r0; c < T.r1; c += kSkCap32) {
      const int n = min(kSkCap32, T.r1 - c);
      __syncthreads();  // the previous chunk has been consumed
      for (int k = tid; k < n; k += kSkThreads) {
        const int2 C = cols[c + k];
        const float4 h = Hi[C.x], l = Lo[C.x], o = boff[C.y];
        float ex, ey, ez, ew;
        float4 hh = make_float4(two_sum(h.x, o.x, ex), two_sum(h.y, o.y, ey), two_sum(h.z, o.z, ez),
                                two_sum(h.w, o.w, ew));
        if constexpr (D <= 3) hh.w = w[c + k];
        else sw[k] = w[c + k];
        shi[k] = hh;
        slo[k] = make_float4(l.x + ex, l.y + ey, l.z + ez, l.w + ew);
      }
      __syncthreads();
      int f = stripe;
      for (; f + S < n; f += 2 * S) {
        const float4 h0 = shi[f], l0 = slo[f], h1 = shi[f + S], l1 = slo[f + S];
        const float w0 = D <= 3 ? h0.w : sw[f], w1 = D <= 3 ? h1.w : sw[f + S];
        a0 = fmaf(f32k<KID>(sqdist2<D>(tha, tla, h0, l0), kc), w0, a0);
        b0 = fmaf(f32k<KID>(sqdist2<D>(thb, tlb, h0, l0), kc), w0, b0);
        a1 = fmaf(f32k<KID>(sqdist2<D>(tha, tla, h1, l1), kc), w1, a1);
        b1 = fmaf(f32k<KID>(sqdist2<D>(thb, tlb, h1, l1), kc), w1, b1);
      }
      if (f < n) {
        const float4 h0 = shi[f], l0 = slo[f];
        const float w0 = D <= 3 ? h0.w : sw[f];
        a0 = fmaf(f32k<KID>(sqdist2<D>(tha, tla, h0, l0), kc), w0, a0);
        b0 = fmaf(f32k<KID>(sqdist2<D>(thb, tlb, h0, l0), kc), w0, b0);
      }
    }
    red[tid] = a0 + a1;
    red2[tid] = b0 + b1;
    __syncthreads();
    if (stripe == 0) {
      float acc_a = 0.f, acc_b = 0.f;
      for (int q = 0; q < S; ++q) {
        acc_a += red[q * G + gi];
        acc_b += red2[q * G + gi];
      }
      float* yl = ylev + (int64_t)(T.level - 1) * N + T.a0;
      if (va) yl[gi] = kscale * acc_a;
      if (vb) yl[gi + G] = kscale * acc_b;
    }
    __syncthreads();  // red and the staging arrays are reused by the next task
  }
}

// ---------------------------------------------------------------- FP64 form --

template <int D>
__device__ __forceinline__ double sqdist64(const double* a, const double* b) {
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const double t = a[k] - b[k];
    s = fma(t, t, s);
  }
  return s;
}

// FP64 pivot rows: the same task lists; coordinates are the tree-order FP64
// points (SoA d x N), so no frames or offsets.
template <int D>
__global__ void __launch_bounds__(kSkThreads)
    k_skel_rows64(const SkTask* __restrict__ tasks, int64_t ntask, const int4* __restrict__ rows,
                  const double* __restrict__ pts, int64_t N, const double* __restrict__ xt, int kid, double kc,
                  double kscale, double* __restrict__ s, double* __restrict__ part) {
  __shared__ double sx[D][kSkCap64];
  __shared__ double sw[kSkCap64];
  __shared__ double red[kSkThreads], red2[kSkThreads];
  const int tid = threadIdx.x;
  for (int64_t it = blockIdx.x; it < ntask; it += gridDim.x) {
    const SkTask T = tasks[it];
    const int nr = T.r1 - T.r0;
    const int G = stripe_width(nr);
    const int S = kSkThreads / G;
    const int gi = tid % G, stripe = tid / G;
    const bool va = gi < nr, vb = gi + G < nr;
    double ta[D], tb[D];
    for (int k = 0; k < D; ++k) {
      ta[k] = va ? pts[(int64_t)k * N + rows[T.r0 + gi].x] : 0.0;
      tb[k] = vb ? pts[(int64_t)k * N + rows[T.r0 + gi + G].x] : 0.0;
    }
    __syncthreads();
    for (int k = tid; k < T.n; k += kSkThreads) {
      const int64_t j = T.a0 + k;
      for (int q = 0; q < D; ++q) sx[q][k] = pts[(int64_t)q * N + j];
      sw[k] = xt[j];
    }
    __syncthreads();
    double a = 0.0, b = 0.0;
    for (int f = stripe; f < T.n; f += S) {
      double xs[D];
      for (int q = 0; q < D; ++q) xs[q] = sx[q][f];
      a = fma(f64fast_of_s(kid, sqdist64<D>(ta, xs), kc), sw[f], a);
      b = fma(f64fast_of_s(kid, sqdist64<D>(tb, xs), kc), sw[f], b);
    }
    red[tid] = a;
    red2[tid] = b;
    __syncthreads();
    if (stripe == 0) {
      double acc_a = 0.0, acc_b = 0.0;
      for (int q = 0; q < S; ++q) {
        acc_a += red[q * G + gi];
        acc_b += red2[q * G + gi];
      }
      if (T.pout < 0) {
        if (va) s[rows[T.r0 + gi].y] = kscale * acc_a;
        if (vb) s[rows[T.r0 + gi + G].y] = kscale * acc_b;
      } else {
        if (va) part[T.pout + gi] = acc_a;
        if (vb) part[T.pout + gi + G] = acc_b;
      }
    }
  }
}

template <int D>
__global__ void __launch_bounds__(kSkThreads)
    k_skel_cols64(const SkTask* __restrict__ tasks, int64_t ntask, const int2* __restrict__ cols,
                  const double* __restrict__ pts, int64_t N, const double* __restrict__ w, int kid, double kc,
                  double kscale, double* __restrict__ ylev) {
  __shared__ double sx[D][kSkCap64];
  __shared__ double sw[kSkCap64];
  __shared__ double red[kSkThreads], red2[kSkThreads];
  const int tid = threadIdx.x;
  for (int64_t it = blockIdx.x; it < ntask; it += gridDim.x) {
    const SkTask T = tasks[it];
    const int nr = T.n;
    const int G = stripe_width(nr);
    const int S = kSkThreads / G;
    const int gi = tid % G, stripe = tid / G;
    const bool va = gi < nr, vb = gi + G < nr;
    double ta[D], tb[D];
    for (int k = 0; k < D; ++k) {
      ta[k] = va ? pts[(int64_t)k * N + T.a0 + gi] : 0.0;
      tb[k] = vb ? pts[(int64_t)k * N + T.a0 + gi + G] : 0.0;
    }
    double a = 0.0, b = 0.0;
    for (int c = T.r0; c < T.r1; c += kSkCap64) {
      const int n = min(kSkCap64, T.r1 - c);
      __syncthreads();
      for (int k = tid; k < n; k += kSkThreads) {
        const int2 C = cols[c + k];
        for (int q = 0; q < D; ++q) sx[q][k] = pts[(int64_t)q * N + C.x];
        sw[k] = w[c + k];
      }
      __syncthreads();
      for (int f = stripe; f < n; f += S) {
        double xs[D];
        for (int q = 0; q < D; ++q) xs[q] = sx[q][f];
        a = fma(f64fast_of_s(kid, sqdist64<D>(ta, xs), kc), sw[f], a);
        b = fma(f64fast_of_s(kid, sqdist64<D>(tb, xs), kc), sw[f], b);
      }
    }
    red[tid] = a;
    red2[tid] = b;
    __syncthreads();
    if (stripe == 0) {
      double acc_a = 0.0, acc_b = 0.0;
      for (int q = 0; q < S; ++q) {
        acc_a += red[q * G + gi];
        acc_b += red2[q * G + gi];
      }
      double* yl = ylev + (int64_t)(T.level - 1) * N + T.a0;
      if (va) yl[gi] = kscale * acc_a;
      if (vb) yl[gi + G] = kscale * acc_b;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ shared steps --

// Row groups cut into several source chunks: s[slot] = scale * (sum of the
// chunks' partials in chunk order). One thread per row.
template <class Acc>
__global__ void k_skel_rowsum(const int4* __restrict__ groups, int64_t ngroup, const int4* __restrict__ rows,
                              const Acc* __restrict__ part, Acc kscale, Acc* __restrict__ s) {
  for (int64_t g = blockIdx.x; g < ngroup; g += gridDim.x) {
    const int4 Gp = groups[g];  // {r0, r1, first partial, chunks}
    const int nr = Gp.y - Gp.x;
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      double acc = 0.0;
      for (int q = 0; q < Gp.w; ++q) acc += (double)part[Gp.z + (int64_t)q * nr + r];
      s[rows[Gp.x + r].y] = (Acc)((double)kscale * acc);
    }
  }
}

// w_b = U_b^-1 (L_b^-1 s_b) in FP64, one warp per low-rank block, the vector in
// shared memory. M (column-major p x p) holds L on and below the diagonal and
// the strict upper part of the unit upper triangular U. In place on t.
template <class Acc>
__global__ void __launch_bounds__(32 * kSkSolveWarps)
    k_skel_solve(const int32_t* __restrict__ blist, int64_t nlist, const int32_t* __restrict__ rank,
                 const int64_t* __restrict__ slot0, const int64_t* __restrict__ luoff, const double* __restrict__ LU,
                 Acc* __restrict__ t) {
  extern __shared__ double skv[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* v = skv + (size_t)wib * kSkMaxP;
  const int64_t nwarps = (int64_t)gridDim.x * kSkSolveWarps;
  for (int64_t item = (int64_t)blockIdx.x * kSkSolveWarps + wib; item < nlist; item += nwarps) {
    const int32_t b = blist[item];
    const int p = rank[b];
    Acc* tb = t + slot0[b];
    const double* M = LU + luoff[b];
    for (int k = lane; k < p; k += 32) v[k] = (double)tb[k];
    __syncwarp();
    for (int k = 0; k < p; ++k) {  // forward: L z = s
      const double* col = M + (int64_t)k * p;
      const double zk = v[k] / col[k];
      __syncwarp();
      if (lane == 0) v[k] = zk;
      for (int l = k + 1 + lane; l < p; l += 32) v[l] = fma(-col[l], zk, v[l]);
      __syncwarp();
    }
    for (int k = p - 1; k > 0; --k) {  // backward: U w = z, unit diagonal
      const double* col = M + (int64_t)k * p;
      const double wk = v[k];
      for (int l = lane; l < k; l += 32) v[l] = fma(-col[l], wk, v[l]);
      __syncwarp();
    }
    for (int k = lane; k < p; k += 32) tb[k] = (Acc)v[k];
    __syncwarp();
  }
}

// FP32 form: W_b = U_b^-1 L_b^-1 formed once at the build (FP64), so that a
// product computes w = W s as a small dense matvec instead of two dependent
// triangular sweeps. One warp per block, lane j solving for column j of W
// (forward with L, then backward with the unit upper U), in place in W.
__global__ void k_skel_inv(const int32_t* __restrict__ blist, int64_t nlist, const int32_t* __restrict__ rank,
                           const int64_t* __restrict__ luoff, const double* __restrict__ LU, double* __restrict__ Wm) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < nlist; item += nwarps) {
    const int32_t b = blist[item];
    const int p = rank[b];
    const double* M = LU + luoff[b];
    double* Wb = Wm + luoff[b];
    for (int j = lane; j < p; j += 32) {
      double* z = Wb + (int64_t)j * p;  // column j
      for (int l = 0; l < j; ++l) z[l] = 0.0;
      for (int l = j; l < p; ++l) {  // L z = e_j
        double acc = l == j ? 1.0 : 0.0;
        for (int m = j; m < l; ++m) acc = fma(-M[l + (int64_t)m * p], z[m], acc);
        z[l] = acc / M[l + (int64_t)l * p];
      }
      for (int l = p - 2; l >= 0; --l) {  // U w = z (unit diagonal)
        double acc = z[l];
        for (int m = l + 1; m < p; ++m) acc = fma(-M[l + (int64_t)m * p], z[m], acc);
        z[l] = acc;
      }
    }
  }
}

// w_b = W_b s_b (FP64 arithmetic, FP32 in and out), one warp per block, in
// place on t; lanes own rows, W column-major so a warp reads 32 consecutive
// entries per column.
__global__ void __launch_bounds__(32 * kSkSolveWarps)
    k_skel_wapply(const int32_t* __restrict__ blist, int64_t nlist, const int32_t* __restrict__ rank,
                  const int64_t* __restrict__ slot0, const int64_t* __restrict__ luoff,
                  const double* __restrict__ Wm, float* __restrict__ t) {
  extern __shared__ double skv[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* v = skv + (size_t)wib * kSkMaxP;
  const int64_t nwarps = (int64_t)gridDim.x * kSkSolveWarps;
  for (int64_t item = (int64_t)blockIdx.x * kSkSolveWarps + wib; item < nlist; item += nwarps) {
    const int32_t b = blist[item];
    const int p = rank[b];
    float* tb = t + slot0[b];
    const double* Wb = Wm + luoff[b];
    for (int k = lane; k < p; k += 32) v[k] = (double)tb[k];
    __syncwarp();
    for (int l0 = 0; l0 < p; l0 += 32) {
      const int l = l0 + lane;
      double acc = 0.0;
      if (l < p) {
        const double* col = Wb + l;
        int k = 0;
        double acc2 = 0.0;
        for (; k + 1 < p; k += 2) {
          acc = fma(col[(int64_t)k * p], v[k], acc);
          acc2 = fma(col[(int64_t)(k + 1) * p], v[k + 1], acc2);
        }
        if (k < p) acc = fma(col[(int64_t)k * p], v[k], acc);
        acc += acc2;
      }
      if (l < p) tb[l] = (float)acc;
    }
    __syncwarp();
  }
}

// Skeleton rank of each low-rank block: the leading terms whose pivot |L(q, q)|
// = |u_q(sigma_q)| stays at least theta times the largest pivot before it.
__global__ void k_skel_trunc(int64_t nblk, const int32_t* __restrict__ rank, const int32_t* __restrict__ bm,
                             const int64_t* __restrict__ toff, const int64_t* __restrict__ uoff,
                             const int32_t* __restrict__ sig, const double* __restrict__ U64, double theta,
                             int32_t* __restrict__ keep) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += (int64_t)gridDim.x * blockDim.x) {
    const int p = rank[b];
    const int64_t m = bm[b];
    int k = 0;
    double big = 0.0;
    for (; k < p; ++k) {
      const double piv = fabs(U64[uoff[b] + (int64_t)k * m + sig[toff[b] + k]]);
      big = fmax(big, piv);
      if (!(piv >= theta * big) || piv == 0.0) break;
    }
    keep[b] = k;
  }
}

// M_b from the ACA factors over the kept leading terms (p' of them):
// M(l, q) = u_q(sigma_l) for l >= q, v_l(tau_q) for l < q.
__global__ void k_skel_lu(const int32_t* __restrict__ blist, int64_t nlist, const int32_t* __restrict__ rank,
                          const int32_t* __restrict__ bm, const int32_t* __restrict__ bn,
                          const int64_t* __restrict__ toff, const int64_t* __restrict__ uoff,
                          const int64_t* __restrict__ voff, const int64_t* __restrict__ luoff,
                          const int32_t* __restrict__ sig, const int32_t* __restrict__ tau,
                          const double* __restrict__ U64, const double* __restrict__ V64, double* __restrict__ LU) {
  for (int64_t item = blockIdx.x; item < nlist; item += gridDim.x) {
    const int32_t b = blist[item];
    const int p = rank[b];
    const int64_t m = bm[b], n = bn[b], t0 = toff[b];
    const double* U = U64 + uoff[b];
    const double* V = V64 + voff[b];
    double* M = LU + luoff[b];
    for (int64_t e = threadIdx.x; e < (int64_t)p * p; e += blockDim.x) {
      const int l = (int)(e % p), q = (int)(e / p);
      M[e] = l >= q ? U[(int64_t)q * m + sig[t0 + l]] : V[(int64_t)l * n + tau[t0 + q]];
    }
  }
}

int grid_of(int64_t n, int cap) { return (int)std::max<int64_t>(1, std::min<int64_t>(n, cap)); }

}  // namespace

// Keeps sigma, tau (already on the device) and the LU factors of K(sigma, tau)
// of every low-rank block (over its kept leading terms); the factor arrays
// themselves are not kept.
int build_skeleton(hodlrdd_s* h, const DevBuf<double>& U64, const DevBuf<double>& V64,
                   const std::vector<int64_t>& uoff64, const std::vector<int64_t>& voff64) {
  const int64_t nblk = h->nblk;
  Plan& P = h->plan;
  cudaStream_t st = h->st;
  h->h_toff.assign(nblk + 1, 0);
  h->factor_elems = 0;
  for (int64_t b = 0; b < nblk; ++b) {
    if (h->h_rank[b] > kSkMaxP) {
      set_error("skeleton form: a block rank exceeds 1024");
      return HODLRDD_ERR_UNSUPPORTED;
    }
    h->h_toff[b + 1] = h->h_toff[b] + h->h_rank[b];
    h->factor_elems += (int64_t)h->h_rank[b] * (h->h_bm[b] + h->h_bn[b]);
  }
  DevBuf<int64_t> du, dv;
  HD_TRY(upload(du, uoff64, st));
  HD_TRY(upload(dv, voff64, st));
  // skeleton ranks: every term in FP64, the leading resolvable terms in FP32
  const double theta = h->opt.precision == HODLRDD_PREC_FP64 ? 0.0 : kSkTheta32;
  HD_TRY(P.sk_rank.alloc(std::max<int64_t>(nblk, 1)));
  if (nblk > 0) {
    k_skel_trunc<<<grid_of((nblk + 255) / 256, 152 * 16), 256, 0, st>>>(nblk, h->rank.p, h->bm.p, h->toff.p, du.p,
                                                                        h->piv_sigma.p, U64.p, theta, P.sk_rank.p);
    HD_CUDA(cudaGetLastError());
  }
  HD_TRY(download(P.h_sk_rank, P.sk_rank.p, (size_t)nblk, st));
  HD_CUDA(cudaStreamSynchronize(st));
  P.h_sk_toff.assign(nblk + 1, 0);
  std::vector<int64_t> luoff(nblk + 1, 0);
  std::vector<int32_t> blist;
  for (int64_t b = 0; b < nblk; ++b) {
    const int pk = P.h_sk_rank[b];
    P.h_sk_toff[b + 1] = P.h_sk_toff[b] + pk;
    luoff[b + 1] = luoff[b] + (int64_t)pk * pk;
    if (pk > 0) blist.push_back((int32_t)b);
  }
  P.sk_terms = P.h_sk_toff[nblk];
  HD_TRY(upload(P.sk_toff, P.h_sk_toff, st));
  HD_TRY(upload(P.sk_luoff, luoff, st));
  HD_TRY(upload(P.sk_blist, blist, st));
  HD_TRY(P.sk_lu.alloc(std::max<int64_t>(luoff[nblk], 1)));
  if (!blist.empty()) {
    k_skel_lu<<<grid_of((int64_t)blist.size(), 152 * 64), 128, 0, st>>>(
        P.sk_blist.p, (int64_t)blist.size(), P.sk_rank.p, h->bm.p, h->bn.p, h->toff.p, du.p, dv.p, P.sk_luoff.p,
        h->piv_sigma.p, h->piv_tau.p, U64.p, V64.p, P.sk_lu.p);
    HD_CUDA(cudaGetLastError());
  }
  if (theta > 0.0 && !blist.empty()) {  // FP32 form: keep W = U^-1 L^-1 instead of L and U
    DevBuf<double> Wm;
    HD_TRY(Wm.alloc(std::max<int64_t>(luoff[nblk], 1)));
    k_skel_inv<<<grid_of(((int64_t)blist.size() + 3) / 4, 152 * 64), 128, 0, st>>>(
        P.sk_blist.p, (int64_t)blist.size(), P.sk_rank.p, P.sk_luoff.p, P.sk_lu.p, Wm.p);
    HD_CUDA(cudaGetLastError());
    HD_CUDA(cudaStreamSynchronize(st));
    P.sk_lu = std::move(Wm);
  }
  HD_CUDA(cudaStreamSynchronize(st));  // du, dv go out of scope
  h->factor_bytes = (int64_t)(P.sk_lu.bytes() + h->piv_sigma.bytes() + h->piv_tau.bytes());
  return HODLRDD_OK;
}

// Task lists of the three steps. Needs the tree, the blocks, the pivots and,
// for the FP32 form, the per-level hi + lo coordinates (build_plan).
int build_skeleton_plan(hodlrdd_s* h) {
  Plan& P = h->plan;
  const int d = h->d;
  const bool f64 = h->opt.precision == HODLRDD_PREC_FP64;
  const int cap = f64 ? kSkCap64 : kSkCap32;
  cudaStream_t st = h->st;
  const int64_t nblk = h->nblk;
  std::vector<int32_t> sig, tau;
  HD_TRY(download(sig, h->piv_sigma.p, (size_t)std::max<int64_t>(h->total_rank, 0), st));
  HD_TRY(download(tau, h->piv_tau.p, (size_t)std::max<int64_t>(h->total_rank, 0), st));
  HD_CUDA(cudaStreamSynchronize(st));
  // per block: (c_J - c_I) h_l, exact in FP32 (|c_J - c_I| <= 3, h_l has 20 significant bits)
  std::vector<float4> boff(std::max<int64_t>(nblk, 1), make_float4(0.f, 0.f, 0.f, 0.f));
  auto coords = [&](int l, int64_t box, int64_t* c) {
    const uint64_t key = h->lv[l].h_bkey[box];
    for (int k = 0; k < d; ++k) {
      c[k] = 0;
      for (int bit = 0; bit < l; ++bit) c[k] |= (int64_t)((key >> (d * bit + k)) & 1u) << bit;
    }
  };
  // columns by slot, and per level the source box -> blocks transpose
  std::vector<int2> cols(std::max<int64_t>(P.sk_terms, 1), make_int2(0, 0));
  std::vector<SkTask> ctask, rtask;
  std::vector<int4> rows, rsum;
  int64_t parts = 0;
  P.sk_pairs = 0;
  for (int l = 1; l <= h->kappa; ++l) {
    const Level& L = h->lv[l];
    const int64_t b0 = h->h_blk_off[l], b1 = h->h_blk_off[l + 1];
    for (int64_t b = b0; b < b1; ++b) {
      const int p = P.h_sk_rank[b];
      if (p == 0) continue;
      int64_t cI[kMaxDim], cJ[kMaxDim];
      coords(l, h->h_bti[b], cI);
      coords(l, h->h_bsj[b], cJ);
      float v[4] = {0.f, 0.f, 0.f, 0.f};
      for (int k = 0; k < d && k < 4; ++k) v[k] = (float)((double)(cJ[k] - cI[k]) * P.h_box[l]);
      boff[b] = make_float4(v[0], v[1], v[2], v[3]);
      for (int q = 0; q < p; ++q)
        cols[P.h_sk_toff[b] + q] = make_int2(h->h_bJ0[b] + tau[h->h_toff[b] + q], (int32_t)b);
      P.sk_pairs += (int64_t)p * (h->h_bm[b] + h->h_bn[b]);
    }
    // column tasks: per target box, its blocks' slots are consecutive
    for (int64_t i = 0; i < L.nb; ++i) {
      const int64_t e0 = b0 + L.h_iloff[i], e1 = b0 + L.h_iloff[i + 1];
      const int64_t s0 = P.h_sk_toff[e0], s1 = P.h_sk_toff[e1];
      if (s1 == s0) continue;
      const int32_t I0 = L.h_bstart[i], m = L.h_bstart[i + 1] - I0;
      for (int32_t r = 0; r < m; r += kSkRows)
        ctask.push_back(SkTask{I0 + r, std::min(kSkRows, m - r), (int32_t)s0, (int32_t)s1, l, -1, 0, 0});
    }
    // row tasks: per source box, the pivot rows of every block reading it
    std::vector<std::vector<int64_t>> by_src(L.nb);
    for (int64_t b = b0; b < b1; ++b)
      if (P.h_sk_rank[b] > 0) by_src[h->h_bsj[b]].push_back(b);
    for (int64_t j = 0; j < L.nb; ++j) {
      if (by_src[j].empty()) continue;
      const int32_t r_first = (int32_t)rows.size();
      for (int64_t b : by_src[j])
        for (int q = 0; q < P.h_sk_rank[b]; ++q)
          rows.push_back(make_int4(h->h_bI0[b] + sig[h->h_toff[b] + q], (int32_t)(P.h_sk_toff[b] + q), (int32_t)b, 0));
      const int32_t r_last = (int32_t)rows.size();
      const int32_t J0 = L.h_bstart[j], nJ = L.h_bstart[j + 1] - J0;
      const int32_t nq = (nJ + cap - 1) / cap;
      for (int32_t r0 = r_first; r0 < r_last; r0 += kSkRows) {
        const int32_t r1 = std::min(r0 + kSkRows, r_last);
        if (nq == 1) {
          rtask.push_back(SkTask{J0, nJ, r0, r1, l, -1, 0, 0});
          continue;
        }
        if (parts + (int64_t)nq * (r1 - r0) >= INT32_MAX) {
          set_error("skeleton form: too many partial sums");
          return HODLRDD_ERR_UNSUPPORTED;
        }
        for (int32_t q = 0; q < nq; ++q)
          rtask.push_back(SkTask{J0 + q * cap, std::min(cap, nJ - q * cap), r0, r1, l,
                                 (int32_t)(parts + (int64_t)q * (r1 - r0)), 0, 0});
        rsum.push_back(make_int4(r0, r1, (int32_t)parts, nq));
        parts += (int64_t)nq * (r1 - r0);
      }
    }
  }
  // coarse levels (larger tasks) were appended first; keep that order
  HD_TRY(upload(P.sk_rtask, rtask, st));
  HD_TRY(upload(P.sk_rsum, rsum, st));
  HD_TRY(upload(P.sk_rows, rows, st));
  HD_TRY(upload(P.sk_ctask, ctask, st));
  HD_TRY(upload(P.sk_cols, cols, st));
  HD_TRY(upload(P.sk_boff, boff, st));
  P.sk_parts = parts;
  HD_TRY(P.sk_part.alloc((size_t)std::max<int64_t>(parts, 1) * (f64 ? 8 : 4)));
  if (!f64) {
    std::vector<const float4*> hp(h->kappa + 1, nullptr), lp(h->kappa + 1, nullptr);
    for (int l = 1; l <= h->kappa; ++l) {
      if (l < (int)P.hi4.size()) {
        hp[l] = P.hi4[l].p;
        lp[l] = P.lo4[l].p;
      }
    }
    for (const SkTask& T : rtask)
      if (!hp[T.level]) {
        set_error("skeleton form: missing level coordinates");
        return HODLRDD_ERR_INVALID;
      }
    HD_TRY(upload(P.sk_hi, hp, st));
    HD_TRY(upload(P.sk_lo, lp, st));
  }
  HD_CUDA(cudaStreamSynchronize(st));
  P.sk_bytes = (int64_t)(P.sk_lu.bytes() + P.sk_luoff.bytes() + P.sk_blist.bytes() + P.sk_rank.bytes() +
                         P.sk_toff.bytes() + P.sk_rtask.bytes() +
                         P.sk_rsum.bytes() + P.sk_rows.bytes() + P.sk_ctask.bytes() + P.sk_cols.bytes() +
                         P.sk_boff.bytes() + P.sk_part.bytes() + h->piv_sigma.bytes() + h->piv_tau.bytes());
  return HODLRDD_OK;
}

namespace {

template <int D, int KID>
void rows32_k(hodlrdd_s* h, cudaStream_t st, const float* xt, float* t) {
  const Plan& P = h->plan;
  const int64_t n = (int64_t)P.sk_rtask.n;
  k_skel_rows<D, KID><<<grid_of(n, INT32_MAX), kSkThreads, 0, st>>>(
      P.sk_rtask.p, n, P.sk_rows.p, P.sk_boff.p, P.sk_hi.p, P.sk_lo.p, xt, (float)kernel_const(h->K),
      (float)h->K.scale, t, reinterpret_cast<float*>(P.sk_part.p));
}
template <int D, int KID>
void cols32_k(hodlrdd_s* h, cudaStream_t st, const float* t, float* ylev) {
  const Plan& P = h->plan;
  const int64_t n = (int64_t)P.sk_ctask.n;
  k_skel_cols<D, KID><<<grid_of(n, INT32_MAX), kSkThreads, 0, st>>>(
      P.sk_ctask.p, n, P.sk_cols.p, P.sk_boff.p, P.sk_hi.p, P.sk_lo.p, t, (float)kernel_const(h->K),
      (float)h->K.scale, ylev, h->N);
}

template <bool ROWS, int D>
void launch32_d(hodlrdd_s* h, cudaStream_t st, const float* in, float* out) {
#define HD_SK_CASE(K)                                       \
  case K:                                                   \
    if constexpr (ROWS) rows32_k<D, K>(h, st, in, out);     \
    else cols32_k<D, K>(h, st, in, out);                    \
    break;
  switch (h->K.id) {
    HD_SK_CASE(HODLRDD_K_LOG)
    HD_SK_CASE(HODLRDD_K_INV_R)
    HD_SK_CASE(HODLRDD_K_MATERN32)
    HD_SK_CASE(HODLRDD_K_GAUSS)
    HD_SK_CASE(HODLRDD_K_EXP)
    HD_SK_CASE(HODLRDD_K_INV_R2_4D)
    HD_SK_CASE(HODLRDD_K_R)
    HD_SK_CASE(HODLRDD_K_SIN)
    default:
      if constexpr (ROWS) rows32_k<D, HODLRDD_K_INV_SQRT1P>(h, st, in, out);
      else cols32_k<D, HODLRDD_K_INV_SQRT1P>(h, st, in, out);
      break;
  }
#undef HD_SK_CASE
}

template <bool ROWS>
void launch32(hodlrdd_s* h, cudaStream_t st, const float* in, float* out) {
  switch (h->d) {
    case 1: launch32_d<ROWS, 1>(h, st, in, out); break;
    case 2: launch32_d<ROWS, 2>(h, st, in, out); break;
    case 3: launch32_d<ROWS, 3>(h, st, in, out); break;
    default: launch32_d<ROWS, 4>(h, st, in, out); break;
  }
}

template <bool ROWS, int D>
void launch64_d(hodlrdd_s* h, cudaStream_t st, const double* in, double* out) {
  const Plan& P = h->plan;
  const double kc = kernel_const(h->K);
  if constexpr (ROWS) {
    const int64_t n = (int64_t)P.sk_rtask.n;
    k_skel_rows64<D><<<grid_of(n, INT32_MAX), kSkThreads, 0, st>>>(
        P.sk_rtask.p, n, P.sk_rows.p, h->pts64.p, h->N, in, h->K.id, kc, h->K.scale, out,
        reinterpret_cast<double*>(P.sk_part.p));
  } else {
    const int64_t n = (int64_t)P.sk_ctask.n;
    k_skel_cols64<D><<<grid_of(n, INT32_MAX), kSkThreads, 0, st>>>(P.sk_ctask.p, n, P.sk_cols.p, h->pts64.p, h->N,
                                                                    in, h->K.id, kc, h->K.scale, out);
  }
}

template <bool ROWS>
void launch64(hodlrdd_s* h, cudaStream_t st, const double* in, double* out) {
  switch (h->d) {
    case 1: launch64_d<ROWS, 1>(h, st, in, out); break;
    case 2: launch64_d<ROWS, 2>(h, st, in, out); break;
    case 3: launch64_d<ROWS, 3>(h, st, in, out); break;
    default: launch64_d<ROWS, 4>(h, st, in, out); break;
  }
}

template <class Acc>
int rows_and_solve(hodlrdd_s* h, cudaStream_t st, const Acc* xt, Acc* t) {
  const Plan& P = h->plan;
  if (P.sk_rtask.n > 0) {
    if constexpr (std::is_same<Acc, double>::value) launch64<true>(h, st, xt, t);
    else launch32<true>(h, st, xt, t);
    h->launches += 1;
  }
  if (P.sk_rsum.n > 0) {
    k_skel_rowsum<Acc><<<grid_of((int64_t)P.sk_rsum.n, 152 * 32), 128, 0, st>>>(
        P.sk_rsum.p, (int64_t)P.sk_rsum.n, P.sk_rows.p, reinterpret_cast<const Acc*>(P.sk_part.p),
        (Acc)h->K.scale, t);
    h->launches += 1;
  }
  if (P.sk_blist.n > 0) {
    const int64_t nl = (int64_t)P.sk_blist.n;
    const size_t smem = (size_t)kSkSolveWarps * kSkMaxP * sizeof(double);
    const int grid = grid_of((nl + kSkSolveWarps - 1) / kSkSolveWarps, 152 * 16);
    if constexpr (std::is_same<Acc, double>::value)
      k_skel_solve<Acc><<<grid, 32 * kSkSolveWarps, smem, st>>>(P.sk_blist.p, nl, P.sk_rank.p, P.sk_toff.p,
                                                                P.sk_luoff.p, P.sk_lu.p, t);
    else
      k_skel_wapply<<<grid, 32 * kSkSolveWarps, smem, st>>>(P.sk_blist.p, nl, P.sk_rank.p, P.sk_toff.p,
                                                            P.sk_luoff.p, P.sk_lu.p, t);
    h->launches += 1;
  }
  HD_CUDA(cudaGetLastError());
  return HODLRDD_OK;
}

}  // namespace

// s = K(sigma, J) x(J) for every low-rank block, then w = U^-1 L^-1 s in place
// on t (slots by block, as the stored form's t vector).
int launch_skeleton_rows(hodlrdd_s* h, cudaStream_t st, const void* xt, void* t) {
  if (h->opt.precision == HODLRDD_PREC_FP64)
    return rows_and_solve<double>(h, st, static_cast<const double*>(xt), static_cast<double*>(t));
  return rows_and_solve<float>(h, st, static_cast<const float*>(xt), static_cast<float*>(t));
}

// ylev[(l - 1) N + i] = sum over the low-rank IL blocks of i's box at level l
// of K(x_i, x_tau) w; rows of boxes without low-rank blocks are left as they are.
int launch_skeleton_cols(hodlrdd_s* h, cudaStream_t st, const void* t, void* ylev) {
  const Plan& P = h->plan;
  if (P.sk_ctask.n == 0) return HODLRDD_OK;
  if (h->opt.precision == HODLRDD_PREC_FP64)
    launch64<false>(h, st, static_cast<const double*>(t), static_cast<double*>(ylev));
  else
    launch32<false>(h, st, static_cast<const float*>(t), static_cast<float*>(ylev));
  h->launches += 1;
  HD_CUDA(cudaGetLastError());
  return HODLRDD_OK;
}

}  // namespace hd
