// ReLU arc-cosine map (stax.Relu in the Appendix A listings) on the device.
// Two FP32 evaluations of J are provided (asin form below, and the
// (1-c)^{3/2} form the kernels use).
//
// For a centred Gaussian pair with variances q, q' and covariance K,
//   E[relu(u) relu(v)] = sqrt(q q') / (2 pi) * J(c),  c = K / sqrt(q q'),
//   J(c) = sqrt(1 - c^2) + c (pi - arccos c).
// Writing J(c) = pi c / 2 + g(c) with the even function
//   g(c) = sqrt(1 - c^2) + |c| asin|c|
// and using asin|c| = pi/2 - asin(sqrt(1 - c^2)) when |c| > sqrt(1 - c^2),
// only asin(m) with m = min(|c|, sqrt(1 - c^2)) in [0, 1/sqrt 2] is needed.
// asin(m) = m + m^3 P(m^2) with P of degree 6, fitted by
// csrc/fit_asin.py (near-minimax, Lawson re-weighted least squares;
// relative error 1.5e-8 in float64, FP32 rounding dominates on the device).
// J is well conditioned at |c| -> 1 (dJ/dc = pi - arccos c is bounded and
// dJ/dsqrt(1-c^2) vanishes there), so FP32 suffices for the map itself.
#pragma once

#include <math.h>

#define NK_PI_F 3.14159265358979323846f
#define NK_HALF_PI_F 1.57079632679489661923f
#define NK_PI_D 3.14159265358979323846
#define NK_INV_2PI_D 0.15915494309189533577

__device__ __forceinline__ float nk_sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// asin(m) for m in [0, 1/sqrt(2)].
__device__ __forceinline__ float nk_asin_small(float m) {
  const float z = m * m;
  float p = 1.112414098e-01f;
  p = fmaf(p, z, -9.249696326e-02f);
  p = fmaf(p, z, 7.689475858e-02f);
  p = fmaf(p, z, 1.641334877e-02f);
  p = fmaf(p, z, 4.649848860e-02f);
  p = fmaf(p, z, 7.488511025e-02f);
  p = fmaf(p, z, 1.666690495e-01f);
  return fmaf(m * z, p, m);
}

// Second form used by the kernels: J(c) = pi c + (1 - c)^{3/2} B(c) on
// [0, 1], B a degree-5 polynomial fitted by csrc/fit_jpos.py (max absolute
// error of J 2.5e-8 in float64, below FP32 rounding of J in [1, pi]).  One
// square root and 8 FMA-pipe operations.  Correlations after a ReLU layer
// are >= 0 (a sum of non-negative terms), so every layer but the first uses
// this form; the first uses J(c) = J(|c|) + pi min(c, 0).
__device__ __forceinline__ float nk_B_poly(float c) {
  float p = -7.025579042e-04f;
  p = fmaf(p, c, 2.948344719e-03f);
  p = fmaf(p, c, -7.401106535e-03f);
  p = fmaf(p, c, 1.875308504e-02f);
  p = fmaf(p, c, -7.079342243e-02f);
  p = fmaf(p, c, 9.999999749e-01f);
  return p;
}

// J(c) for c >= 0 (values above 1 are clamped).
__device__ __forceinline__ float nk_J01_f32(float c) {
  c = fminf(c, 1.f);
  const float u = 1.f - c;
  const float w3 = u * nk_sqrt_approx(u);
  return fmaf(w3, nk_B_poly(c), NK_PI_F * c);
}

// J(c) in FP32 for any c (clamped to [-1, 1]).
__device__ __forceinline__ float nk_J_f32(float c) {
  const float a = fminf(fabsf(c), 1.f);
  const float u = 1.f - a;
  const float w3 = u * nk_sqrt_approx(u);
  const float j = fmaf(w3, nk_B_poly(a), NK_PI_F * a);
  return fmaf(NK_PI_F, fmaxf(fminf(c, 0.f), -1.f), j);
}

// The asin-based form of J(c) (kept as an independent second evaluation for
// tests): J(c) = pi c/2 + sqrt(1-c^2) + |c| asin|c| with the range reduction.
__device__ __forceinline__ float nk_J_asin_f32(float c) {
  c = fminf(fmaxf(c, -1.f), 1.f);
  const float om = fmaf(-c, c, 1.f);
  const float sn = nk_sqrt_approx(om);
  const float a = fabsf(c);
  const float m = fminf(a, sn);
  const float as = nk_asin_small(m);
  const float t = (a > sn) ? (NK_HALF_PI_F - as) : as;
  const float g = fmaf(a, t, sn);
  return fmaf(c, NK_HALF_PI_F, g);
}

// J'(c) = pi - arccos(c) in FP32 (used by the adjoint).
__device__ __forceinline__ float nk_dJ_f32(float c) {
  c = fminf(fmaxf(c, -1.f), 1.f);
  const float om = fmaf(-c, c, 1.f);
  const float sn = nk_sqrt_approx(om);
  const float a = fabsf(c);
  const float m = fminf(a, sn);
  const float as = nk_asin_small(m);
  // pi - acos(c) = pi/2 + asin(c)
  const float asa = (a > sn) ? (NK_HALF_PI_F - as) : as;  // asin|c|
  return NK_HALF_PI_F + copysignf(asa, c);
}

// asin(c) in FP32 for c in [-1, 1] (clamped): asin|c| = asin_small(|c|) for
// |c| <= 1/sqrt(2), else pi/2 - asin_small(sqrt(1 - c^2)); the sign of c.
// The Erf map's argument 2K / sqrt((m + 2q)(m' + 2q')) stays below
// 2q / (1 + 2q) < 1 in magnitude, where asin is well conditioned.
__device__ __forceinline__ float nk_asin_f32(float c) {
  c = fminf(fmaxf(c, -1.f), 1.f);
  const float a = fabsf(c);
  const float sn = nk_sqrt_approx(fmaf(-c, c, 1.f));
  const float m = fminf(a, sn);
  const float as = nk_asin_small(m);
  return copysignf((a > sn) ? (NK_HALF_PI_F - as) : as, c);
}

// Erf map in FP64: E[erf(u) erf(v)] = (2/pi) asin(2 K / sqrt((1 + 2 q1)(1 + 2 q2)))
// for centred Gaussians with variances q1, q2 and covariance K.
__device__ __forceinline__ double nk_erf_map_f64(double K, double q1, double q2) {
  double c = 2.0 * K / sqrt((1.0 + 2.0 * q1) * (1.0 + 2.0 * q2));
  c = fmin(fmax(c, -1.0), 1.0);
  return (2.0 / NK_PI_D) * asin(c);
}

// J(c) and J'(c) = pi - arccos c together, from one arcsine: J' = pi/2 +
// asin c and J = sqrt(1 - c^2) + c J' (the adjoint needs both).  Near c = -1
// the two terms of J cancel to (1 + c)^{3/2}; the absolute error stays at
// FP32 rounding of sqrt(1 - c^2), which is what the adjoint's products see.
__device__ __forceinline__ void nk_J_dJ_f32(float c, float& J, float& dJ) {
  c = fminf(fmaxf(c, -1.f), 1.f);
  const float sn = nk_sqrt_approx(fmaf(-c, c, 1.f));
  const float a = fabsf(c);
  const float as = nk_asin_small(fminf(a, sn));
  dJ = NK_HALF_PI_F + copysignf((a > sn) ? (NK_HALF_PI_F - as) : as, c);
  J = fmaf(c, dJ, sn);
}

// J(c) in FP64 with the CUDA double-precision arccos.
__device__ __forceinline__ double nk_J_f64(double c) {
  c = fmin(fmax(c, -1.0), 1.0);
  return sqrt(fmax(1.0 - c * c, 0.0)) + c * (NK_PI_D - acos(c));
}

// Full map in FP64: Kt = sqrt(q1 q2)/(2 pi) J(K / sqrt(q1 q2)), 0 if q1 q2 == 0.
__device__ __forceinline__ double nk_relu_map_f64(double K, double q1, double q2) {
  const double s = sqrt(q1 * q2);
  if (!(s > 0.0)) return 0.0;
  return s * NK_INV_2PI_D * nk_J_f64(K / s);
}
