// The inference kernels' GELU (Sec. 2.2 activation, exact form v Phi(v)), evaluated
// without erf: see gelu_poly below.
#pragma once

#include <cuda_runtime.h>

#include "gelu_poly.cuh"

namespace lbmfno {

// GELU(v) = v Phi(v) = max(v, 0) - a Q(a) with a = |v| and Q(a) = Phi(-a) =
// exp(-a^2 / 2) S(a), S(a) = erfcx(a / sqrt 2) / 2 evaluated as a degree-7 polynomial in
// u = a / 3 - 1 (gelu_poly.cuh, fitted by gelu_fit.py on a in [0, 6]); a is clamped to 6:
// beyond it the exact a Q(a) is below 6e-9 and the clamped value, 1.1e-7, stands in for it.
// Absolute error within 5e-6 (1 + |v|) of the exact GELU (the activation is rounded to
// bfloat16 right after, a relative step of 2^-8),
// NaN propagates, GELU(+inf) = +inf.  max(v, 0) is the NaN-propagating max.NaN (an ALU
// instruction, which leaves the FP32 pipes to the polynomial), so that a NaN input is
// not turned into 0.
__device__ __forceinline__ float gelu_poly(float v) {
  constexpr float c[GELU_S_DEG + 1] = GELU_S_COEFFS;
  const float a = fminf(fabsf(v), 6.0f);
  const float u = fmaf(a, 1.0f / 3.0f, -1.0f);
  float p = c[GELU_S_DEG];
#pragma unroll
  for (int k = GELU_S_DEG - 1; k >= 0; --k) p = fmaf(p, u, c[k]);
  float e;  // exp(-a^2 / 2) = 2^(-a^2 log2(e) / 2)
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(a * a * -0.72134752044448170f));
  float h;
  asm("max.NaN.f32 %0, %1, 0f00000000;" : "=f"(h) : "f"(v));
  return fmaf(-a, e * p, h);
}

// Two activations at once with packed FP32 arithmetic: the same operations in the same
// order as gelu_poly, so each lane's result is identical to gelu_poly's.
__device__ __forceinline__ float2 gelu_poly2(float2 v) {
  constexpr float c[GELU_S_DEG + 1] = GELU_S_COEFFS;
  const float2 a = make_float2(fminf(fabsf(v.x), 6.0f), fminf(fabsf(v.y), 6.0f));
  const float2 u = __ffma2_rn(a, make_float2(1.0f / 3.0f, 1.0f / 3.0f), make_float2(-1.0f, -1.0f));
  float2 p = make_float2(c[GELU_S_DEG], c[GELU_S_DEG]);
#pragma unroll
  for (int k = GELU_S_DEG - 1; k >= 0; --k) p = __ffma2_rn(p, u, make_float2(c[k], c[k]));
  const float2 t = __fmul2_rn(__fmul2_rn(a, a), make_float2(-0.72134752044448170f, -0.72134752044448170f));
  float2 e;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.x) : "f"(t.x));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.y) : "f"(t.y));
  float2 h;
  asm("max.NaN.f32 %0, %1, 0f00000000;" : "=f"(h.x) : "f"(v.x));
  asm("max.NaN.f32 %0, %1, 0f00000000;" : "=f"(h.y) : "f"(v.y));
  return __ffma2_rn(make_float2(-a.x, -a.y), __fmul2_rn(e, p), h);
}

}  // namespace lbmfno
