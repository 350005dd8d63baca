// Pair arithmetic shared by the on-the-fly kernels (near field, direct sum,
// skeleton apply): FP32 kernel functions of the squared distance and the
// squared distance of two points held as box-relative FP32 hi + lo pairs.
#pragma once

#include "internal.cuh"

namespace hd {
namespace {

// Hardware reciprocal (square root) approximations, PTX rsqrt / rcp
// .approx.ftz (relative error below 2^-22); the packed path treats squared
// distances below the smallest normal FP32 number as coincident points.
__device__ __forceinline__ float rsqrt_hw(float s) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(s));
  return r;
}
__device__ __forceinline__ float rcp_hw(float s) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(s));
  return r;
}
constexpr float kTinySq = 1.17549435e-38f;  // smallest normal FP32 number

__device__ __forceinline__ float sqrt_hw(float s) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(s));
  return r;
}

// Kernel functions of r = sqrt(s) for the packed near field: hardware
// approximations for square roots and reciprocals, the CUDA fast exponential
// (__expf) for the exponential kernels.
template <int KID>
__device__ __forceinline__ float f32k(float s, float c) {
  if constexpr (KID == HODLRDD_K_LOG) return s == 0.0f ? 0.0f : 0.5f * logf(s);
  else if constexpr (KID == HODLRDD_K_INV_R) return s < kTinySq ? 0.0f : rsqrt_hw(s);
  else if constexpr (KID == HODLRDD_K_MATERN32) {
    const float a = c * sqrt_hw(s);
    return (1.0f + a) * __expf(-a);
  } else if constexpr (KID == HODLRDD_K_GAUSS) return __expf(-c * s);
  else if constexpr (KID == HODLRDD_K_EXP) return __expf(-c * sqrt_hw(s));
  else if constexpr (KID == HODLRDD_K_INV_R2_4D) return s < kTinySq ? 0.0f : c * rcp_hw(s);
  else if constexpr (KID == HODLRDD_K_R) return sqrt_hw(s);
  else if constexpr (KID == HODLRDD_K_SIN) return sinf(sqrt_hw(s));
  else return rsqrt_hw(1.0f + sqrt_hw(s));
}

// a += F(s) w with F = f32k<KID>. For the kernels that are zero at r = 0 the
// value is left out by a predicated multiply-add (s below the smallest normal
// number: a coincident point) instead of a select of zero: one instruction less
// per pair, the same sums (a + 0 w = a).
template <int KID>
__device__ __forceinline__ void acc_pair(float s, float c, float w, float& a) {
  if constexpr (KID == HODLRDD_K_INV_R || KID == HODLRDD_K_INV_R2_4D || KID == HODLRDD_K_LOG) {
    float f;
    if constexpr (KID == HODLRDD_K_INV_R) f = rsqrt_hw(s);
    else if constexpr (KID == HODLRDD_K_INV_R2_4D) f = c * rcp_hw(s);
    else f = 0.5f * logf(s);
    const float lim = KID == HODLRDD_K_LOG ? 0.0f : kTinySq;
    if constexpr (KID == HODLRDD_K_LOG)
      asm("{\n\t.reg .pred p;\n\tsetp.gt.f32 p, %1, %2;\n\t@p fma.rn.f32 %0, %3, %4, %0;\n\t}"
          : "+f"(a) : "f"(s), "f"(lim), "f"(f), "f"(w));
    else
      asm("{\n\t.reg .pred p;\n\tsetp.ge.f32 p, %1, %2;\n\t@p fma.rn.f32 %0, %3, %4, %0;\n\t}"
          : "+f"(a) : "f"(s), "f"(lim), "f"(f), "f"(w));
  } else {
    a = fmaf(f32k<KID>(s, c), w, a);
  }
}

// 1/sqrt(s) to about one ulp: the hardware approximation refined by one Newton
// step, y1 = y0 + y0 (1 - s y0^2) / 2, with the residual formed by an FMA.
__device__ __forceinline__ float rsqrt_nt(float s) {
  const float y0 = rsqrt_hw(s);
  const float e = fmaf(-s, y0 * y0, 1.0f);
  return fmaf(0.5f * y0, e, y0);
}

// The same kernel functions to about one ulp (the Newton-refined reciprocal
// square root, the IEEE square root and division, the CUDA expf / logf / sinf)
// for the skeleton apply's pivot-row step, whose rounding is amplified by the
// interpolation operator.
template <int KID>
__device__ __forceinline__ float f32k_rn(float s, float c) {
  if constexpr (KID == HODLRDD_K_LOG) return s == 0.0f ? 0.0f : 0.5f * logf(s);
  else if constexpr (KID == HODLRDD_K_INV_R) return s < kTinySq ? 0.0f : rsqrt_nt(s);
  else if constexpr (KID == HODLRDD_K_MATERN32) {
    const float a = c * sqrtf(s);
    return (1.0f + a) * expf(-a);
  } else if constexpr (KID == HODLRDD_K_GAUSS) return expf(-c * s);
  else if constexpr (KID == HODLRDD_K_EXP) return expf(-c * sqrtf(s));
  else if constexpr (KID == HODLRDD_K_INV_R2_4D) return s < kTinySq ? 0.0f : c / s;
  else if constexpr (KID == HODLRDD_K_R) return sqrtf(s);
  else if constexpr (KID == HODLRDD_K_SIN) return sinf(sqrtf(s));
  else return rsqrt_nt(1.0f + sqrtf(s));
}

// a + b = s + e exactly (Knuth's two-sum).
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
  return s;
}

// Squared distance from the high parts alone (kernels smooth in r^2).
template <int D>
__device__ __forceinline__ float sqdist1(const float4& th, const float4& sh) {
  float t = th.x - sh.x;
  float s = t * t;
  if (D > 1) {
    t = th.y - sh.y;
    s = fmaf(t, t, s);
  }
  if (D > 2) {
    t = th.z - sh.z;
    s = fmaf(t, t, s);
  }
  if (D > 3) {
    t = th.w - sh.w;
    s = fmaf(t, t, s);
  }
  return s;
}

template <int D>
__device__ __forceinline__ float sqdist2(const float4& th, const float4& tl, const float4& sh, const float4& sl) {
  float t = (th.x - sh.x) + (tl.x - sl.x);
  float s = t * t;
  if (D > 1) {
    t = (th.y - sh.y) + (tl.y - sl.y);
    s = fmaf(t, t, s);
  }
  if (D > 2) {
    t = (th.z - sh.z) + (tl.z - sl.z);
    s = fmaf(t, t, s);
  }
  if (D > 3) {
    t = (th.w - sh.w) + (tl.w - sl.w);
    s = fmaf(t, t, s);
  }
  return s;
}

}  // namespace
}  // namespace hd
