// expm1_poly.h -- written by gen_expm1_poly.py (do not edit).
// expm1(r) ~ r p(r) on [-0.35, 0.35], p interpolating (e^r - 1)/r at the Chebyshev
// points; coefficients rounded to double; p(r) by Horner's rule, one FMA per coefficient.
#pragma once
#include <cuda_runtime.h>
namespace sco {
constexpr double kExpLn2 = 0.6931471805599453;  // ln 2, rounded
constexpr double kExpInvLn2 = 1.4426950408889634;  // 1 / ln 2, rounded
// expm1_poly: degree 8; max relative error of r p(r) in exact arithmetic with these
// coefficients, on 40001 points: 9.76e-14
__host__ __device__ __forceinline__ double expm1_poly(double r) {
  double p = 2.762645049050251e-06;
  p = fma(p, r, 2.487764798531672e-05);
  p = fma(p, r, 0.00019841206303368908);
  p = fma(p, r, 0.0013888818977515853);
  p = fma(p, r, 0.00833333335495731);
  p = fma(p, r, 0.041666666904604285);
  p = fma(p, r, 0.16666666666646798);
  p = fma(p, r, 0.4999999999978138);
  p = fma(p, r, 1.0);
  return p;
}
// expm1_poly6: degree 6; max relative error of r p(r) in exact arithmetic with these
// coefficients, on 40001 points: 2.85e-10
__host__ __device__ __forceinline__ double expm1_poly6(double r) {
  double p = 0.00019900428151915095;
  p = fma(p, r, 0.0013942147844205415);
  p = fma(p, r, 0.008333297083738308);
  p = fma(p, r, 0.04166634028910043);
  p = fma(p, r, 0.16666666722181583);
  p = fma(p, r, 0.5000000049985063);
  p = fma(p, r, 1.0);
  return p;
}
}  // namespace sco
