// Float-float ("double-single") arithmetic on the FP32 pipes: a value is an
// unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2, about
// 48 significant bits. Built from the error-free transformations of Dekker and
// Knuth (TwoSum, Fast2Sum, TwoProduct through a fused multiply-add), with the
// elementary functions the kernels need written from their definitions:
// Newton steps from the hardware reciprocal square root, a 64-entry table of
// 2^(j/64) for exp, and one Newton step on exp for log. Every operation that
// feeds an error-free transformation uses the _rn intrinsics so the compiler
// cannot contract it into a fused multiply-add.
//
// Accuracy (relative, for the arguments the near field passes): rsqrt, sqrt,
// reciprocal about 2^-44; exp about 2^-45; log about 2^-45 absolute. The tests
// compare every kernel function against FP64 references.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace hd {

struct ff {
  float h, l;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ ff ff_fast(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = ff_two_sum(a.h, b.h);
  return ff_fast(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ ff ff_addf(ff a, float b) {
  const ff s = ff_two_sum(a.h, b);
  return ff_fast(s.h, __fadd_rn(s.l, a.l));
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  ff p = ff_prod(a.h, b.h);
  p.l = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l));
  return ff_fast(p.h, p.l);
}

__device__ __forceinline__ ff ff_mulf(ff a, float b) {
  ff p = ff_prod(a.h, b);
  p.l = __fmaf_rn(a.l, b, p.l);
  return ff_fast(p.h, p.l);
}

__device__ __forceinline__ ff ff_from_double(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1 / sqrt(a), a > 0: y + y (1 - a y^2) / 2 with the residual in float-float.
__device__ __forceinline__ ff ff_rsqrt(ff a) {
  const float y = rsqrt_approx(a.h);
  const ff y2 = ff_prod(y, y);
  const ff z = ff_prod(a.h, y2.h);
  const float zl = __fmaf_rn(a.h, y2.l, __fmaf_rn(a.l, y2.h, z.l));
  const float t = __fsub_rn(__fsub_rn(1.0f, z.h), zl);  // 1 - z.h is exact (z.h near 1)
  return ff_fast(y, __fmul_rn(__fmul_rn(y, t), 0.5f));
}

// sqrt(a), a >= 0: s + (a - s^2) / (2 s) from s = a rsqrt(a).
__device__ __forceinline__ ff ff_sqrt(ff a) {
  if (a.h <= 0.0f) return {0.0f, 0.0f};
  const float y = rsqrt_approx(a.h);
  const float s = __fmul_rn(a.h, y);
  const ff p = ff_prod(s, s);
  const float d = __fadd_rn(__fsub_rn(__fsub_rn(a.h, p.h), p.l), a.l);
  return ff_fast(s, __fmul_rn(__fmul_rn(d, y), 0.5f));
}

// 1 / a, a != 0: y + y (1 - a y).
__device__ __forceinline__ ff ff_recip(ff a) {
  const float y = rcp_approx(a.h);
  const ff z = ff_prod(a.h, y);
  const float t = __fsub_rn(__fsub_rn(1.0f, z.h), __fmaf_rn(a.l, y, z.l));
  return ff_fast(y, __fmul_rn(y, t));
}

// Constants of exp, set by the host from the mathematics (ff_exp_const):
// ln2/64 in three pieces (the first with 11 significant bits, so that n times
// it is exact for |n| < 2^13), 64/ln2, and 2^(j/64) = t[j].h + t[j].l. Kernels
// copy t into shared memory and pass it to ff_exp.
struct FfExpConst {
  float c0, c1, c2;  // ln2 / 64 = c0 + c1 + c2
  float inv;         // 64 / ln2, rounded
  ff t[64];          // 2^(j / 64)
};

struct FfExp {
  float c0, c1, c2, inv;
  const ff* t;  // 64 entries (shared memory)
};

// exp(a) for |a.h| <= 87 (0 below -87, where the FP64 value is under 2^-125):
// a = n ln2 / 64 + r with |r| <= ln2 / 128, exp(r) from its Taylor series to
// r^5 (the terms from r^3 in FP32), times 2^(j/64) from the table and 2^(n / 64)
// by exponent.
__device__ __forceinline__ ff ff_exp(ff a, const FfExp& K) {
  if (a.h < -87.0f) return {0.0f, 0.0f};
  const float n = rintf(__fmul_rn(a.h, K.inv));
  const float r0 = __fmaf_rn(-n, K.c0, a.h);  // exact
  const ff t1 = ff_prod(n, K.c1);
  ff r = ff_two_sum(r0, -t1.h);
  r.l = __fadd_rn(r.l, __fadd_rn(a.l, __fsub_rn(-t1.l, __fmul_rn(n, K.c2))));
  r = ff_fast(r.h, r.l);
  // exp(r) = 1 + qp, qp = r + r^2/2 + r^3 (1/6 + r/24 + r^2/120): r^2/2 (up to
  // 2^-16) keeps its float-float low part, the terms from r^3 (up to 2^-25) are
  // summed in FP32, and 1 + qp is formed last so that the low part of the result
  // carries no term larger than ulp(1)
  const ff r2 = ff_prod(r.h, r.h);
  const float tail = __fmul_rn(__fmul_rn(r2.h, r.h),
                               __fmaf_rn(r.h, __fmaf_rn(r.h, 1.0f / 120.0f, 1.0f / 24.0f), 1.0f / 6.0f));
  const ff half_r2 = {__fmul_rn(0.5f, r2.h),
                      __fadd_rn(__fmul_rn(0.5f, r2.l), __fadd_rn(__fmul_rn(r.h, r.l), tail))};
  const ff qp = ff_add(r, half_r2);
  ff e = ff_two_sum(1.0f, qp.h);
  e = ff_fast(e.h, __fadd_rn(e.l, qp.l));
  const int ni = (int)n;
  const int j = ni & 63;
  const int q = (ni - j) / 64;  // floor(n / 64)
  e = ff_mul(e, K.t[j]);
  // 2^q in two steps so that neither factor overflows or is subnormal
  const int q1 = q / 2, q2 = q - q1;
  const float s1 = __int_as_float((q1 + 127) << 23), s2 = __int_as_float((q2 + 127) << 23);
  return {__fmul_rn(__fmul_rn(e.h, s1), s2), __fmul_rn(__fmul_rn(e.l, s1), s2)};
}

// log(a), a > 0: y = log(a) in FP32, then y + u - u^2 / 2 with u = a e^-y - 1.
// u is about ulp(y), up to 2^-19 for |y| near 30, so it stays a float-float
// (p.h - 1 exact, plus p.l) and only the u^2 / 2 term is rounded in FP32.
__device__ __forceinline__ ff ff_log(ff a, const FfExp& K) {
  const float y = logf(a.h);
  const ff e = ff_exp({-y, 0.0f}, K);
  const ff p = ff_mul(a, e);
  const float uh = __fsub_rn(p.h, 1.0f);  // exact (p.h near 1)
  const ff s = ff_two_sum(y, uh);
  return ff_fast(s.h, __fadd_rn(s.l, __fsub_rn(p.l, __fmul_rn(__fmul_rn(uh, uh), 0.5f))));
}

}  // namespace hd
