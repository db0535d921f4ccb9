// sco_device.cuh -- device-side building blocks of the SCO library (sm_103a):
// counter-based random numbers, the spin proposal, the dipolar pair energy,
// double-double arithmetic for near-tie decisions, and the kernel parameter block.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "expm1_poly.h"
#include "log_table.h"

namespace sco {

// Philox counter word 3 per use of the random stream (the library's stream layout).
constexpr uint64_t kTagInit = 1, kTagSwitch = 2, kTagPropose = 3;
// Bit 31 of a CSR entry: nearest-neighbour exchange bond whose dipolar pair was switched off.
constexpr uint32_t kExchOnly = 0x80000000u;
constexpr uint32_t kIndexMask = 0x7FFFFFFFu;

// Parameters every kernel reads (passed by value).
struct DevParams {
  int32_t Lx, Ly;
  int64_t N;        // Lx * Ly
  int64_t K;        // half-plane displacement count
  double J, D, beta, bD;  // beta = fl(1/T), bD = fl(beta * D)
  double inv_bD58;        // fl(2^58 / bD): exponential draw -> hazard prefix units
  float inv_bD58_f;       // its FP32 rounding
  float beta_f;           // fl32(beta), for the FP32 screens (no FP64 operation there)
  float bJ_f;             // fl32(fl(beta J))
  int switching;          // 1 when beta D > 0 (pairs can be switched off)
  uint64_t key0, key1;    // Philox key: seed, replica
  double ln2_hi, ln2_lo;  // ln 2 as a double-double
  unsigned long long lx_magic;  // floor((2^64 - 1) / Lx) + 1 (0 when Lx = 1)
};

// floor(u / d) for 32-bit u and d >= 2 by one 64-bit high multiply with
// M = floor((2^64 - 1) / d) + 1 (Lemire, Kaser and Kurz, "Faster remainder by direct
// computation", 2019); M = 0 stands for d = 1.
__host__ __device__ __forceinline__ unsigned long long div_magic(unsigned long long d) {
  return d > 1 ? 0xFFFFFFFFFFFFFFFFull / d + 1ull : 0ull;
}
__device__ __forceinline__ uint32_t div_by_magic(uint32_t u, unsigned long long M) {
  return M ? (uint32_t)__umul64hi(M, (unsigned long long)u) : u;
}

// Row y = i / Lx of site i, keeping 64-bit integer division out of the inner loops.
__device__ __forceinline__ uint32_t site_row(uint32_t i, const DevParams& P) {
  return div_by_magic(i, P.lx_magic);
}

// Warp sum (lane 0 receives the total).
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------------------
// Philox4x64-10, Salmon, Moraes, Dror and Shaw (SC'11): two 64x64->128 multiplies per round
// on counter words 0 and 2, high halves mixed with words 1, 3 and the key, key bumped by
// the Weyl increments after every round.
struct W4 {
  uint64_t w[4];
};

__device__ __forceinline__ W4 philox(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                     uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t B0 = 0x9E3779B97F4A7C15ull, B1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += B0;
    k1 += B1;
  }
  W4 o;
  o.w[0] = c0; o.w[1] = c1; o.w[2] = c2; o.w[3] = c3;
  return o;
}

// m 2^-53 for an integer 0 <= m <= 2^53, built from its bits (integer operations only, exact;
// 64-bit integer conversions would run on the FP64 pipe).
__device__ __forceinline__ double scaled53(uint64_t m) {
  if (m == 0) return 0.0;
  const int e = 63 - __clzll((long long)m);  // m in [2^e, 2^(e+1)), e <= 53
  const uint64_t mant = e <= 52 ? (m << (52 - e)) & 0xFFFFFFFFFFFFFull : 0ull;
  return __longlong_as_double((long long)(((uint64_t)(e - 53 + 1023) << 52) | mant));
}
__device__ __forceinline__ double u53(uint64_t w) { return scaled53(w >> 11); }
__device__ __forceinline__ double u53pos(uint64_t w) { return scaled53((w >> 11) + 1); }

// 2 u - 1 for u = u53(w): with m = w >> 11, fl(fl(2u) - 1) is the exact (m - 2^52) 2^-52
// (|m - 2^52| <= 2^52 needs no rounding; +0 when 2u = 1), built from its bits.
__device__ __forceinline__ double centred53(uint64_t w) {
  const long long d = (long long)(w >> 11) - (1ll << 52);
  if (d == 0) return 0.0;
  const uint64_t mag = (uint64_t)(d < 0 ? -d : d);  // <= 2^52
  const int e = 63 - __clzll((long long)mag);
  const uint64_t mant = (mag << (52 - e)) & 0xFFFFFFFFFFFFFull;
  const uint64_t b = ((uint64_t)(e - 52 + 1023) << 52) | mant;
  return __longlong_as_double((long long)(d < 0 ? b | 0x8000000000000000ull : b));
}

// 2 v for a normal or zero v (exact: one more in the exponent field).
__device__ __forceinline__ double twice(double v) {
  const long long b = __double_as_longlong(v);
  return (b & 0x7FFFFFFFFFFFFFFFll) == 0 ? v : __longlong_as_double(b + (1ll << 52));
}

// Marsaglia (1972): reject unless 0 < s = a1^2 + a2^2 < 1, then
// S = (2 a1 sqrt(1-s), 2 a2 sqrt(1-s), 1 - 2s), a = 2u - 1.  Each operation rounded on its own
// so that the spin is the same bit pattern on every IEEE machine; the doublings are exact, so
// fl(fl(2 a1) h) = 2 fl(a1 h) and fl(1 - fl(2 s)) = fma(-2, s, 1).  Split in two so that a loop
// over attempts can take the square root once, after it.
__device__ __forceinline__ bool marsaglia_point(uint64_t w0, uint64_t w1, double& a1, double& a2,
                                                double& s) {
  a1 = centred53(w0);
  a2 = centred53(w1);
  s = __dadd_rn(__dmul_rn(a1, a1), __dmul_rn(a2, a2));
  const unsigned long long sb = (unsigned long long)__double_as_longlong(s);  // s >= +0
  return sb != 0ull && sb < 0x3FF0000000000000ull;
}
__device__ __forceinline__ void marsaglia_spin(double a1, double a2, double s, double& x,
                                               double& y, double& z) {
  const double h = __dsqrt_rn(__dsub_rn(1.0, s));
  x = twice(__dmul_rn(a1, h));
  y = twice(__dmul_rn(a2, h));
  z = __fma_rn(-2.0, s, 1.0);
}
__device__ __forceinline__ bool marsaglia(uint64_t w0, uint64_t w1, double& x, double& y,
                                          double& z) {
  double a1, a2, s;
  if (!marsaglia_point(w0, w1, a1, a2, s)) return false;
  marsaglia_spin(a1, a2, s, x, y, z);
  return true;
}

// c(r^2) = fl(1 / fl(fl(r2 r2) fl(sqrt r2))): the FP64 constant standing for r^-5.
__device__ __forceinline__ double coupling_c(int64_t r2) {
  const double q = (double)r2;
  return __ddiv_rn(1.0, __dmul_rn(__dmul_rn(q, q), __dsqrt_rn(q)));
}

// A(r^2) = trunc(fl(fl(2^60 / fl(r2 sqrt r2)) (1 + 2^-50))) + 1 > 2^60 / r^3, so that
// V_max = D A 2^-59 >= 2D / r^3, the maximum of the dipolar pair energy.
__device__ __forceinline__ uint64_t hazard_A(int64_t r2) {
  const double q = (double)r2;
  const double t = __ddiv_rn(0x1p60, __dmul_rn(q, __dsqrt_rn(q)));
  return __double2ull_rz(__dmul_rn(t, 1.0 + 0x1p-50)) + 1ull;
}

// Dipolar pair energy of Eq. (6) with c ~ r^-5 and d = (dx, dy, 0):
// V = D c [r^2 (S_i.S_j) - 3 (S_i.d)(S_j.d)].  |error| <= 2^-47 |D| c r^2 with or without FMA.
__device__ __forceinline__ double pair_V(double Dc, double r2, double ax, double ay, double az,
                                         double bx, double by, double bz, double fx, double fy) {
  const double ss = ax * bx + ay * by + az * bz;
  const double pa = ax * fx + ay * fy;
  const double pb = bx * fx + by * fy;
  return Dc * (r2 * ss - 3.0 * (pa * pb));
}

// The library's own expm1 for x <= 0.35, branch-free (a warp never runs two versions): x =
// k ln2 + r with k = round(x / ln2) (by the 1.5 2^52 shift) and r = fma(-k, ln2, x),
// expm1(r) = r p(r) (p of expm1_poly.h, interpolation error < 1e-13), expm1(x) =
// fma(2^k, expm1(r), 2^k - 1), which rounds to -1 exactly below x = -40 (e^x < 2^-57; k is
// clamped at -1000 so that 2^k stays normal).  Relative error below
// 2^-43: interpolation 2^-43.2; Horner <= gamma_16 p(|r|) / p(r) <= 23 u; r off by at most
// |k| |ln2 - fl(ln2)| <= 58 x 2.3e-17; for k <= -1 the 2^k expm1(r) part (<= 0.42 2^k) carries
// these while |expm1(x)| >= 0.29.  Stated as kExpm1RelErr = 2^-42; the FP64 decisions carry it
// in their error bounds.
constexpr double kExpm1RelErr = 0x1p-42;
// The same with p of degree 6 (expm1_poly6, interpolation error < 2.9e-10): relative error below
// 2^-31.6 by the same argument; stated as kExpm1RelErr6 = 2^-31.  For the sweep decisions, whose
// bound adds these errors relatively (the switch's survival margin is absolute and keeps the
// accurate one: next to the thinning bound of a far pair it must stay small).
constexpr double kExpm1RelErr6 = 0x1p-31;
template <int kDeg>
__device__ __forceinline__ double expm1_np_deg(double x) {
  const double t = fma(x, kExpInvLn2, 0x1.8p52);
  const double kd = t - 0x1.8p52;
  const int k = max(__double2loint(t), -1000);
  const double r = fma(-kd, kExpLn2, x);
  const double e = r * (kDeg == 8 ? expm1_poly(r) : expm1_poly6(r));
  const double s = __longlong_as_double((long long)(1023 + k) << 52);
  // below x = -40 (k <= -58, s (1 + e) < 2^-57) this rounds to -1 exactly, the clamp of k keeping
  // s normal; no select for that range (one FP64 instruction)
  return fma(s, e, s - 1.0);
}
__device__ __forceinline__ double expm1_np(double x) { return expm1_np_deg<8>(x); }

// The library's own natural logarithm for normal 0 < x <= 1 (table-driven after Tang, ACM TOMS
// 16(4), 1990; table and coefficients in log_table.h): x = 2^k m, m in [sqrt(2)/2, sqrt(2)), F =
// 1 + j/256 nearest to m (j and F from the bits), r = (m - F) / F with |r| < 0.0028 (m - F
// exact), log x = k ln2 + log F + log1p(r), log1p(r) = r + r^2 q(r), q of degree 4 (truncation
// below 2^-53.5 |r|).  Relative error below 2^-50: r off by 2^-52 relative, the polynomial by a
// few ulp of r, the sums by an ulp of |k ln2 + log F| <= 3.6 |log x| (the worst case k = 0,
// F != 1, where |log F| >= 0.0039 > |r|).  Stated as kLogRelErr = 2^-49.  13 FP64 operations.
constexpr double kLogRelErr = 0x1p-49;
__device__ __forceinline__ double log_np(double x) {
  const long long xb = __double_as_longlong(x);
  int k = (int)((xb >> 52) & 0x7FF) - 1023;
  const long long frac = xb & 0xFFFFFFFFFFFFFll;
  const bool big = frac >= 0x6A09E667F3BCDll;  // m = 1.frac >= sqrt(2): halve it
  k += big ? 1 : 0;
  const double m = __longlong_as_double(frac | (big ? 0x3FE0000000000000ll : 0x3FF0000000000000ll));
  // j = round((m - 1) 256): for m in [1, 2) round(frac 2^-44); for m/2 round(frac 2^-45) - 128
  const int j = big ? (int)(((frac >> 44) + 1) >> 1) - 128 : (int)(((frac >> 43) + 1) >> 1);
  const long long fb = j >= 0 ? (0x3FF0000000000000ll | ((long long)j << 44))
                              : (0x3FE0000000000000ll | ((long long)(128 + j) << 45));
  const double* t = kLogTab[j - kLogJmin];
  const double inv = __ldg(t), lh = __ldg(t + 1), ll = __ldg(t + 2);
  const double r = (m - __longlong_as_double(fb)) * inv;
  const double q = fma(fma(fma(fma(kLogC6, r, kLogC5), r, kLogC4), r, kLogC3), r, kLogC2);
  const double lp = fma(r * r, q, r);
  const double kd = (double)k;
  return fma(kd, kLogLn2Hi, lh) + (lp + fma(kd, kLogLn2Lo, ll));
}
__device__ __forceinline__ double expm1_np6(double x) { return expm1_np_deg<6>(x); }
// -expm1_np6(x) formed directly: -(s e + (s - 1)) = (1 - s) - s e is one FMA with the sign folded
// into its operands; round to nearest is symmetric, so the value is exactly -expm1_np6(x) (one
// FP64 negation fewer where the term is stored and multiplied).
__device__ __forceinline__ double neg_expm1_np6(double x) {
  const double t = fma(x, kExpInvLn2, 0x1.8p52);
  const double kd = t - 0x1.8p52;
  const int k = max(__double2loint(t), -1000);
  const double r = fma(-kd, kExpLn2, x);
  const double e = r * expm1_poly6(r);
  const double s = __longlong_as_double((long long)(1023 + k) << 52);
  return fma(-s, e, 1.0 - s);
}

// Sweep constants of a pair at (|dx|, |dy|) for the FP64 decisions (64 bytes).  With the
// signs of (dx, dy) applied to a3x, a3y, ax, ay, the field of S_j on site i scaled by beta is
// f = a1 S_j - (S_j . (a3x, a3y)) (dx, dy, 0), so x = beta (V - Vmax) = S_i . f - bvm.
struct __align__(64) Sw64 {
  double a1;        // fl(beta fl(Dc r^2))
  double a3x, a3y;  // fl(fl(beta fl(3 Dc)) |dx|), fl(fl(beta fl(3 Dc)) |dy|)
  double ax, ay;    // |dx|, |dy|
  double bvm;       // fl(beta Vmax)
  double c0;        // bound on |error of x| not scaling with |x|, plus 2^-52 (2 beta Vmax)
  double bsw;       // margin bound of the FP64 survival test of the switch (see table.cu)
};

// x with its sign flipped when neg (bit operation, no FP64 instruction)
__device__ __forceinline__ double flip_if(double x, bool neg) {
  return __longlong_as_double(__double_as_longlong(x) ^ ((long long)neg << 63));
}
// x < 0 strictly (not -0), from the bits
__device__ __forceinline__ bool neg_strict(double x) {
  const long long b = __double_as_longlong(x);
  return b < 0 && b != (long long)0x8000000000000000ull;
}
// bits of a double >= 0, ordered like its value
__device__ __forceinline__ unsigned long long pos_bits(double x) {
  return (unsigned long long)__double_as_longlong(x);
}
// a signed integer ordered like the value of a (non-NaN) double: ord(a) < ord(b) iff a < b
// (the two zeros map to 0 and -1; no FP64 instruction)
__device__ __forceinline__ long long ord_bits(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 ? b : (long long)(0x8000000000000000ull - (unsigned long long)b) - 1;
}
// biased exponent field of a double >= 0 (x >= 2^(e - 1023) for normal x; 0 for zero and
// subnormals, which then read as tiny)
__device__ __forceinline__ int exp_field(double x) {
  return (int)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF;
}

// ---------------------------------------------------------------------------------------
// Double-double arithmetic (Dekker 1971; Knuth's two-sum; Hida, Li and Bailey's QD layout)
// for re-evaluating decisions whose FP64 margin is inside its error bound.
struct dd {
  double hi, lo;
};

__host__ __device__ __forceinline__ dd two_sum(double a, double b) {
  const double s = a + b;
  const double bb = s - a;
  const double e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__host__ __device__ __forceinline__ dd quick_two_sum(double a, double b) {
  const double s = a + b;
  return {s, b - (s - a)};
}
__host__ __device__ __forceinline__ dd two_prod(double a, double b) {
  const double p = a * b;
#ifdef __CUDA_ARCH__
  return {p, __fma_rn(a, b, -p)};
#else
  return {p, __builtin_fma(a, b, -p)};
#endif
}
__host__ __device__ __forceinline__ dd dd_from(double a) { return {a, 0.0}; }
__host__ __device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
__host__ __device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }
__host__ __device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
__host__ __device__ __forceinline__ dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return quick_two_sum(p.hi, p.lo);
}
__host__ __device__ __forceinline__ dd dd_mul_d(dd a, double b) {
  dd p = two_prod(a.hi, b);
  p.lo += a.lo * b;
  return quick_two_sum(p.hi, p.lo);
}
__host__ __device__ __forceinline__ dd dd_div(dd a, dd b) {
  const double q1 = a.hi / b.hi;
  dd r = dd_sub(a, dd_mul_d(b, q1));
  const double q2 = r.hi / b.hi;
  r = dd_sub(r, dd_mul_d(b, q2));
  const double q3 = r.hi / b.hi;
  dd q = quick_two_sum(q1, q2);
  return dd_add(q, dd_from(q3));
}
__host__ __device__ __forceinline__ dd dd_ldexp(dd a, int e) {
#ifdef __CUDA_ARCH__
  return {scalbn(a.hi, e), scalbn(a.lo, e)};
#else
  return {__builtin_scalbn(a.hi, e), __builtin_scalbn(a.lo, e)};
#endif
}
__host__ __device__ __forceinline__ bool dd_lt(dd a, dd b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__host__ __device__ __forceinline__ dd dd_from_u64(uint64_t a) {
  const double hi = (double)(a & ~0x7FFull);  // top bits, exact
  const double lo = (double)(a & 0x7FFull);   // low 11 bits, exact
  return quick_two_sum(hi, lo);
}

// expm1 of a double-double of modulus < 1: x / 2^10, Taylor series, then ten doublings
// t <- 2t + t^2 of e^y - 1 (keeps the relative accuracy near 0).
__host__ __device__ inline dd dd_expm1_small(dd x) {
  const dd y = dd_ldexp(x, -10);
  dd term = y, sum = y;
  for (int n = 2; n <= 14; ++n) {
    // 1/n as a double-double: h = fl(1/n), l = (1 - n h) / n with the residual exact by FMA
    const double h = 1.0 / n;
#ifdef __CUDA_ARCH__
    const dd inv = {h, __fma_rn(-(double)n, h, 1.0) / n};
#else
    const dd inv = {h, __builtin_fma(-(double)n, h, 1.0) / n};
#endif
    term = dd_mul(dd_mul(term, y), inv);
    sum = dd_add(sum, term);
  }
  for (int k = 0; k < 10; ++k) sum = dd_add(dd_ldexp(sum, 1), dd_mul(sum, sum));
  return sum;
}

// exp and expm1 for a double-double: x = k ln2 + r, |r| <= ln2 / 2.
__host__ __device__ inline dd dd_expm1(dd x, dd ln2) {
  if (x.hi > 745.0) return {INFINITY, 0.0};
  if (x.hi < -745.0) return {-1.0, 0.0};
  const double kf = floor(x.hi / ln2.hi + 0.5);
  const int k = (int)kf;
  const dd r = dd_sub(x, dd_mul_d(ln2, kf));
  const dd t = dd_expm1_small(r);
  if (k == 0) return t;
  // 2^k (1 + t) - 1
  return dd_sub(dd_ldexp(dd_add(dd_from(1.0), t), k), dd_from(1.0));
}
__host__ __device__ inline dd dd_exp(dd x, dd ln2) {
  return dd_add(dd_expm1(x, ln2), dd_from(1.0));
}
// log by one Newton step on exp from the FP64 logarithm: x1 = x0 + y e^-x0 - 1.
__host__ __device__ inline dd dd_log(dd y, dd ln2) {
#ifdef __CUDA_ARCH__
  const double x0 = log(y.hi);
#else
  const double x0 = __builtin_log(y.hi);
#endif
  const dd e = dd_exp(dd_from(-x0), ln2);
  const dd c = dd_sub(dd_mul(y, e), dd_from(1.0));
  return dd_add(dd_from(x0), c);
}
// log(1 - e^x) for x < 0 (Maechler 2012 branch point at -ln 2).
__host__ __device__ inline dd dd_log1mexp(dd x, dd ln2) {
  if (x.hi > -ln2.hi) return dd_log(dd_neg(dd_expm1(x, ln2)), ln2);
  return dd_log(dd_sub(dd_from(1.0), dd_exp(x, ln2)), ln2);
}

// V = D c [r^2 (a.b) - 3 (a.d)(b.d)] in double-double from FP64 inputs.
__host__ __device__ inline dd dd_pair_V(double D, double c, double r2, const double* a,
                                        const double* b, double fx, double fy) {
  dd ss = two_prod(a[0], b[0]);
  ss = dd_add(ss, two_prod(a[1], b[1]));
  ss = dd_add(ss, two_prod(a[2], b[2]));
  const dd pa = dd_add(two_prod(a[0], fx), two_prod(a[1], fy));
  const dd pb = dd_add(two_prod(b[0], fx), two_prod(b[1], fy));
  const dd inner = dd_sub(dd_mul_d(ss, r2), dd_mul_d(dd_mul(pa, pb), 3.0));
  return dd_mul(two_prod(D, c), inner);
}

// V_max = D A 2^-59 in double-double.
__host__ __device__ inline dd dd_vmax(double D, uint64_t A) {
  return dd_ldexp(dd_mul_d(dd_from_u64(A), D), -59);
}

}  // namespace sco
