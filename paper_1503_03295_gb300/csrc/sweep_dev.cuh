// sweep_dev.cuh -- per-site decision of step (B) of Sec. 2.1 (Metropolis update under the
// switched Hamiltonian H' of Eq. (4)), shared by the single-lattice and batched sweeps.
//
// Proposal for site i at MC step t: Philox tag PROPOSE, counter (i, t, a); attempt a uses
// words 0, 1 for Marsaglia's sphere point and word 2 of the successful attempt is the
// acceptance uniform u; 64 failed attempts keep the spin.  The move is accepted iff
// u < exp(-beta dE'), i.e. u == 0 or ln u + beta dE' < 0, with
//   beta dE' = sum_{surviving j} [beta V(S', S_j) - L(S') - beta V(S, S_j) + L(S)]
//              - beta J (S' - S) . sum_{nn j} S_j,
//   L = log(1 - exp(beta (V - Vmax)))   (so that beta Vbar = beta V - L, Eq. (3)).
// The decision is taken in FP64 (or FP32 in the FP32-guarded form) with a bound on the
// rounding error of the margin; a site whose margin is inside the bound is settled by one
// warp, in FP64 (after FP32) and then in double-double.
#pragma once

#include <cstdint>

#include "sco_internal.h"

namespace sco {
namespace {

struct SiteCtx {
  int64_t i;
  int32_t xi, yi;
  double S[3], Sn[3];
  double u;
};

// The pseudointeraction terms enter as sum_j [L_o,j - L_n,j] = log(prod z_o) - log(prod z_n)
// with z = 1 - e^x = -expm1(x): one expm1 per pair energy and two logarithms per site (the
// cached FP64 path compares the products instead: u prod z_o e^(sum dx) < prod z_n, see
// accept_fp64_cached).  The products are renormalised by 2^kScale (exact) so that they never
// underflow.
constexpr int kScale64 = 600;
constexpr int kScale32 = 60;

// p by 2^600 on the exponent field when below 2^-600, counted in sc (a multiply would be issued
// on every pair as a select); false for a subnormal or zero p (the decision then goes to the
// exact path).
__device__ __forceinline__ bool renorm600(double& p, int& sc) {
  const unsigned long long b = pos_bits(p);
  if (b >= 0x1A70000000000000ull) return true;  // 2^-600
  if ((b >> 52) == 0) return false;
  p = __longlong_as_double((long long)(b + (600ull << 52)));
  ++sc;
  return true;
}

// Pair terms from the sweep table entry (Sw64): the beta-scaled field of S_j on site i,
// f = a1 S_j - (S_j . a3 d) d, gives x = S.f - bvm = beta V(S) - beta Vmax for the old and the
// new spin (7 + 2 x 3 FP64 operations); where only the proposed spin's term is formed (the pair
// cache holds the old one), x = a1 (S'.S_j) - (S_j.a3 d)(S'.d) - bvm takes 9.  Either way the
// rounding stays far inside c0.
//
// Error bound of the margin mu = ln u + beta dE' (first order, doubled):
//   per pair, |dx| <= c0 + eps_r |x|, and c0 from the table already includes eps_r 2 beta Vmax;
//   z = -expm1(x) has relative error eps_z + |dx| / z;  log of a product of n factors adds
//   n eps_r;  the logarithms eps_f |log P|;  sum (x_new - x_old) adds 2 sum c0 (the x errors)
//   and (n + 2) eps_r sum |x_new - x_old| <= (n + 2) eps_r 2 sum bvm <= (n + 2) sum c0 (c0 >=
//   2^-51 bvm by construction).  The first-order analysis needs lin = sum_j |dx_j| / z_j small:
//   each ratio is below 2^(e(c0_j) - e(z_j) + 1) with e the exponent field, so with two z per
//   pair lin <= n 2^(dmax + 2), dmax the largest exponent difference, found with integer
//   operations; it must stay below 2^-10 or the decision is left undecided.

// FP64 decision (0: reject, 1: accept, 2: undecided).  eps_r = 2^-52 (unit roundoff, with
// margin), eps_f = kLogRelErr for the library's log_np (inputs in (0, 1]), eps_z =
// kExpm1RelErr6 for the library's expm1_np6 (two per pair, doubled: 4 eps_z).  Compares, minima
// and renormalisation tests work on the bits of positive doubles (integer pipe).
__device__ __forceinline__ int accept_fp64(const DevParams& P, const SiteCtx& c,
                                           const Sw64* __restrict__ sw,
                                           const double* __restrict__ s,
                                           const uint32_t* __restrict__ row_ptr,
                                           const uint32_t* __restrict__ col) {
  const double S0 = c.S[0], S1 = c.S[1], S2 = c.S[2];
  const double N0 = c.Sn[0], N1 = c.Sn[1], N2 = c.Sn[2];
  double bdv = 0.0, pz_o = 1.0, pz_n = 1.0;
  unsigned long long c0m = 0;  // bits of the largest c0 (n max c0 bounds their sum)
  int dmax = -2046;  // largest e(c0_j) - e(z_j)
  int sc_o = 0, sc_n = 0, n = 0;
  const uint32_t e1 = row_ptr[c.i + 1];
  for (uint32_t e = row_ptr[c.i]; e < e1; ++e) {
    const uint32_t cj = col[e];
    if (cj & kExchOnly) continue;
    const int64_t j = cj;
    const uint32_t yj = site_row((uint32_t)j, P);
    const int32_t dx = (int32_t)((uint32_t)j - yj * (uint32_t)P.Lx) - c.xi;
    const int32_t dy = (int32_t)yj - c.yi;
    const Sw64& t = sw[(int64_t)(dx < 0 ? -dx : dx) + (int64_t)P.Lx * (dy < 0 ? -dy : dy)];
    const double fx = flip_if(t.ax, dx < 0), fy = flip_if(t.ay, dy < 0);
    const double ax3 = flip_if(t.a3x, dx < 0), ay3 = flip_if(t.a3y, dy < 0);
    const double a1 = t.a1, bvm = t.bvm;
    const double bx = s[j], by = s[P.N + j], bz = s[2 * P.N + j];
    const double tp = bx * ax3 + by * ay3;
    const double gx = a1 * bx - tp * fx;
    const double gy = a1 * by - tp * fy;
    const double gz = a1 * bz;
    // three FMAs each; c0 covers the roundings (those touching bvm stay below 2^-51 bvm)
    const double xn = fma(N0, gx, fma(N1, gy, fma(N2, gz, -bvm)));
    const double xo = fma(S0, gx, fma(S1, gy, fma(S2, gz, -bvm)));
    if (!neg_strict(xn) || !neg_strict(xo)) return 2;
    const double zn = neg_expm1_np6(xn), zo = neg_expm1_np6(xo);
    pz_n *= zn;
    pz_o *= zo;
    if (!renorm600(pz_n, sc_n) || !renorm600(pz_o, sc_o)) return 2;
    bdv += xn - xo;
    dmax = max(dmax, exp_field(t.c0) - min(exp_field(zn), exp_field(zo)));
    c0m = max(c0m, pos_bits(t.c0));
    ++n;
  }
  if (n > 0 && dmax + 2 + (32 - __clz(n)) > -10) return 2;  // n <= 2^(32 - clz n)
  // n 2^(dmax + 2), the power of two from its bits (dmax + 2 <= -10 here; below -1022: 0)
  const double lin = n > 0 && dmax + 2 >= -1022
                         ? (double)n * __longlong_as_double((long long)(dmax + 2 + 1023) << 52)
                         : 0.0;
  double tex = 0.0, bex = 0.0;
  if (P.J != 0.0) {
    double h0 = 0.0, h1 = 0.0, h2 = 0.0;
    const int64_t nb[4] = {c.xi > 0 ? c.i - 1 : -1, c.xi + 1 < P.Lx ? c.i + 1 : -1,
                           c.yi > 0 ? c.i - P.Lx : -1, c.yi + 1 < P.Ly ? c.i + P.Lx : -1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (nb[q] < 0) continue;
      h0 += s[nb[q]];
      h1 += s[P.N + nb[q]];
      h2 += s[2 * P.N + nb[q]];
    }
    const double dot = (c.Sn[0] - c.S[0]) * h0 + (c.Sn[1] - c.S[1]) * h1 + (c.Sn[2] - c.S[2]) * h2;
    tex = -(P.beta * P.J) * dot;
    bex = 0x1p-44 * fabs(P.beta * P.J);
  }
  const double lo = log_np(pz_o), ln = log_np(pz_n);
  // prod z = stored product * 2^(-kScale * count)
  const double scale = (double)((sc_n - sc_o) * kScale64) * P.ln2_hi;
  const double lu = log_np(c.u);
  const double mu = lu + ((bdv + tex) + ((lo - ln) + scale));
  const double c0s = (double)n * __longlong_as_double((long long)c0m);
  const double B = 2.0 * ((double)(n + 4) * c0s + 2.0 * lin + n * (4.0 * kExpm1RelErr6 + 0x1p-51) +
                          kLogRelErr * (fabs(lo) + fabs(ln) + fabs(lu)) + bex +
                          0x1p-51 * (fabs(scale) + fabs(tex) + fabs(bdv) + fabs(mu)));
  if (mu < -B) return 1;
  if (mu > B) return 0;
  return 2;
}

// The pair cache of the FP64 form (single lattice).  For every surviving dipolar pair (half-edge
// id h, carried by both CSR entries of the pair) record keep[h] holds two halves of
// {1 - P = -expm1(x), x = beta (V - Vmax)}, each with the error of any FP64 evaluation of it
// (|x error| <= c0 + 2^-52 |x|, relative error of the elementary function within
// kExpm1RelErr6).  Half p_i ^ p_j holds the pair at the current spins, p_i being the parity of
// site i's accepted moves since the switch (which leaves its FP64 values in the first half) or
// a rebuild (PairCache::upd).  While a site is decided it reads that half and writes the pair
// at its proposed spin into the other one: an acceptance flips its parity and so makes the
// written half the current one, a rejection leaves the read half current.  The endpoint decided
// last writes only when the next MC step keeps the graph.  So per pair endpoint one of the two
// expm1 evaluations and one of the two dot products are read instead of computed, and nothing
// has to be carried between the steps of an epoch.  A written 1 - P <= 0 (the proposed x not
// strictly negative in FP64) makes every reader leave its decision to the double-double path,
// which does not use the cache.

// The site's PairCache::upd byte after its decision: an acceptance flips the parity (bit 2).
__device__ __forceinline__ uint8_t upd_decided(uint32_t ui, bool accepted) {
  return (uint8_t)(accepted ? ((ui & 4u) ^ 4u) | 2u : (ui & 4u) | 1u);
}

// accept_fp64 with the old-spin terms from the pair cache; writes the proposed-spin term of
// every pair (the loop visits every pair, also when the decision is already undecided).
__device__ __forceinline__ int accept_fp64_cached(const DevParams& P, const SiteCtx& c,
                                                  const Sw64* __restrict__ sw,
                                                  const double* __restrict__ s,
                                                  const uint32_t* __restrict__ row_ptr,
                                                  const uint32_t* __restrict__ col,
                                                  const PairCache& pc, uint32_t ui) {
  const double S0 = c.S[0], S1 = c.S[1], S2 = c.S[2];
  const double N0 = c.Sn[0], N1 = c.Sn[1], N2 = c.Sn[2];
  double bdv = 0.0, pz_o = 1.0, pz_n = 1.0;
  unsigned long long c0m = 0;
  int dmax = -2046;
  int sc_o = 0, sc_n = 0, n = 0;
  bool bad = false;
  const uint32_t e1 = row_ptr[c.i + 1];
  for (uint32_t e = row_ptr[c.i]; e < e1; ++e) {
    const uint32_t cj = col[e];
    if (cj & kExchOnly) continue;
    const int64_t j = cj;
    const uint32_t h = pc.hid[e];
    const uint32_t uj = pc.upd[j];
    const uint32_t yj = site_row((uint32_t)j, P);
    const int32_t dx = (int32_t)((uint32_t)j - yj * (uint32_t)P.Lx) - c.xi;
    const int32_t dy = (int32_t)yj - c.yi;
    const Sw64& t = sw[(int64_t)(dx < 0 ? -dx : dx) + (int64_t)P.Lx * (dy < 0 ? -dy : dy)];
    const double fx = flip_if(t.ax, dx < 0), fy = flip_if(t.ay, dy < 0);
    const double ax3 = flip_if(t.a3x, dx < 0), ay3 = flip_if(t.a3y, dy < 0);
    const double a1 = t.a1, bvm = t.bvm;
    const double bx = s[j], by = s[P.N + j], bz = s[2 * P.N + j];
    // {1 - P, x} of the pair at the old spin: one 16-byte read of the record's sector, from
    // the half given by the two parities (j's flipped already if it moved in this step)
    double2* rec = reinterpret_cast<double2*>(&pc.keep[h]);
    const uint32_t hf = ((ui ^ uj) >> 2) & 1u;
    const double2 kv = rec[hf];
    const double zo = kv.x, xo = kv.y;
    // x = a1 (S'.S_j) - (S_j.a3 d)(S'.d) - bvm for the proposed spin S'
    const double ns = N0 * bx + N1 * by + N2 * bz;
    const double tp = bx * ax3 + by * ay3;
    const double nd = N0 * fx + N1 * fy;
    const double xn = fma(a1, ns, fma(-tp, nd, -bvm));
    const bool okn = neg_strict(xn);
    const double zn = okn ? neg_expm1_np6(xn) : -1.0;
    if ((uj & 3u) == 0u || pc.carry) rec[hf ^ 1u] = make_double2(zn, xn);
    // the cached term must be a positive number (a non-positive one marks an FP64 evaluation
    // that could not be trusted)
    if (!okn || !neg_strict(xo) || !(pos_bits(zo) - 1ull < 0x7FEFFFFFFFFFFFFFull)) {
      bad = true;
      continue;
    }
    pz_n *= zn;
    pz_o *= zo;
    if (!renorm600(pz_n, sc_n) || !renorm600(pz_o, sc_o)) bad = true;
    bdv += xn - xo;
    dmax = max(dmax, exp_field(t.c0) - min(exp_field(zn), exp_field(zo)));
    c0m = max(c0m, pos_bits(t.c0));
    ++n;
  }
  if (bad) return 2;
  if (n > 0 && dmax + 2 + (32 - __clz(n)) > -10) return 2;  // n <= 2^(32 - clz n)
  const double lin = n > 0 && dmax + 2 >= -1022
                         ? (double)n * __longlong_as_double((long long)(dmax + 2 + 1023) << 52)
                         : 0.0;
  double tex = 0.0, bex = 0.0;
  if (P.J != 0.0) {
    double h0 = 0.0, h1 = 0.0, h2 = 0.0;
    const int64_t nb[4] = {c.xi > 0 ? c.i - 1 : -1, c.xi + 1 < P.Lx ? c.i + 1 : -1,
                           c.yi > 0 ? c.i - P.Lx : -1, c.yi + 1 < P.Ly ? c.i + P.Lx : -1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (nb[q] < 0) continue;
      h0 += s[nb[q]];
      h1 += s[P.N + nb[q]];
      h2 += s[2 * P.N + nb[q]];
    }
    const double dot = (c.Sn[0] - c.S[0]) * h0 + (c.Sn[1] - c.S[1]) * h1 + (c.Sn[2] - c.S[2]) * h2;
    tex = -(P.beta * P.J) * dot;
    bex = 0x1p-44 * fabs(P.beta * P.J);
  }
  // The decision in product form, without logarithms: mu < 0 is u Pz_o e^A < Pz_n with A = bdv +
  // tex and Pz = pz 2^(-600 sc).  e^A = 2^k e^r, k = round(A / ln2) (|k| <= 2^20, else left
  // undecided), e^r = 1 + r p(r) with p of expm1_np6 (relative error below 2^-32, the reduction's
  // below 2^-34); X = u pz_o e^r and K = k + 600 (sc_n - sc_o), and X 2^K against pz_n is decided
  // on the exponent fields when they differ by 2 or more, else by D = X 2^K - pz_n (X 2^K formed
  // exactly from the bits).  delta bounds the relative errors of X 2^K and pz_n together,
  // doubled: the terms of the logarithmic form's bound without its logarithms, and 2^-31 for e^r,
  // its reduction, the two products and D.
  const double A = bdv + tex;
  const double t = fma(A, kExpInvLn2, 0x1.8p52);
  const double kd = t - 0x1.8p52;
  const int k = __double2loint(t);
  if (k > (1 << 20) || k < -(1 << 20)) return 2;
  const double r = fma(-kd, kExpLn2, A);
  const double er = fma(r, expm1_poly6(r), 1.0);
  const double X = (c.u * pz_o) * er;
  const double c0s = (double)n * __longlong_as_double((long long)c0m);
  const double delta = 2.0 * ((double)(n + 4) * c0s + 2.0 * lin +
                              n * (4.0 * kExpm1RelErr6 + 0x1p-51) + bex +
                              0x1p-51 * (fabs(tex) + fabs(bdv)) + 0x1p-31);
  if (!(delta < 0.25)) return 2;
  const int eX = exp_field(X), eY = exp_field(pz_n);
  if (eX == 0) return 1;  // u = 0
  const int dE = eX + k + kScale64 * (sc_n - sc_o) - eY;
  if (dE >= 2) return 0;   // X 2^K >= 2^(eY + 2) > 2 pz_n
  if (dE <= -2) return 1;  // X 2^K < 2^(eY - 1) <= pz_n / 2
  const double Xs = __longlong_as_double(__double_as_longlong(X) + ((long long)(dE + eY - eX) << 52));
  const double D = Xs - pz_n;
  const long long oD = ord_bits(D), ol = ord_bits(delta * pz_n);
  if (oD < -ol - 1) return 1;  // D < -delta pz_n
  if (oD > ol) return 0;       // D > delta pz_n
  return 2;
}

// FP32 screen of the same decision: shadow spins (|dS| <= 2^-24 per component), FP32 table
// constants, CUDA's single-precision expm1f / logf (<= 1 ulp; 4x margin: eps_f = 2^-21),
// eps_r = 2^-23, and a compensated (Neumaier) sum of the V' - V terms.
__device__ __forceinline__ int accept_fp32(const DevParams& P, const SiteCtx& c,
                                           const float4* __restrict__ sw,
                                           const float4* __restrict__ s32,
                                           const uint32_t* __restrict__ row_ptr,
                                           const uint32_t* __restrict__ col) {
  if (c.u < 0x1p-100) return 2;
  const float beta = P.beta_f;
  const float ax = (float)c.S[0], ay = (float)c.S[1], az = (float)c.S[2];
  const float nx = (float)c.Sn[0], ny = (float)c.Sn[1], nz = (float)c.Sn[2];
  float sum = 0.f, comp = 0.f, sum_abs = 0.f, pz_o = 1.f, pz_n = 1.f, lin = 0.f, c0s = 0.f;
  int sc_o = 0, sc_n = 0, n = 0;
  const uint32_t e1 = row_ptr[c.i + 1];
  for (uint32_t e = row_ptr[c.i]; e < e1; ++e) {
    const uint32_t cj = col[e];
    if (cj & kExchOnly) continue;
    const int64_t j = cj;
    const uint32_t yj = site_row((uint32_t)j, P);
    const int32_t dx = (int32_t)((uint32_t)j - yj * (uint32_t)P.Lx) - c.xi;
    const int32_t dy = (int32_t)yj - c.yi;
    const float4 t =
        __ldg(&sw[(int64_t)(dx < 0 ? -dx : dx) + (int64_t)P.Lx * (dy < 0 ? -dy : dy)]);
    const float4 sj = s32[j];
    const float bx = sj.x, by = sj.y, bz = sj.z;
    const float fx = (float)dx, fy = (float)dy;
    const float tp = t.y * (bx * fx + by * fy);
    const float gx = t.x * bx - tp * fx;
    const float gy = t.x * by - tp * fy;
    const float gz = t.x * bz;
    const float Vn = nx * gx + ny * gy + nz * gz;
    const float Vo = ax * gx + ay * gy + az * gz;
    const float xn = beta * Vn - t.z, xo = beta * Vo - t.z;
    if (!(xn < 0.f) || !(xo < 0.f)) return 2;
    const float zn = -expm1f(xn), zo = -expm1f(xo);
    if (!(zn >= 0x1p-60f) || !(zo >= 0x1p-60f)) return 2;
    // |dx| / z per pair (first order needs it small); FP32 reciprocal, 1.001 for its rounding
    const float ln_ = (t.w + 0x1p-23f * -xn) * (1.001f * __frcp_rn(zn));
    const float lo_ = (t.w + 0x1p-23f * -xo) * (1.001f * __frcp_rn(zo));
    if (!(ln_ <= 0x1p-10f) || !(lo_ <= 0x1p-10f)) return 2;
    lin += ln_ + lo_;
    pz_n *= zn;
    pz_o *= zo;
    if (pz_n < 0x1p-60f) { pz_n *= 0x1p60f; ++sc_n; }
    if (pz_o < 0x1p-60f) { pz_o *= 0x1p60f; ++sc_o; }
    const float dv = Vn - Vo;
    const float tsum = sum + dv;  // Neumaier compensated summation
    comp += fabsf(sum) >= fabsf(dv) ? (sum - tsum) + dv : (dv - tsum) + sum;
    sum = tsum;
    sum_abs += fabsf(dv);
    c0s += t.w;
    ++n;
  }
  float tex = 0.f, bex = 0.f;
  if (P.J != 0.0) {
    float h0 = 0.f, h1 = 0.f, h2 = 0.f;
    const int64_t nb[4] = {c.xi > 0 ? c.i - 1 : -1, c.xi + 1 < P.Lx ? c.i + 1 : -1,
                           c.yi > 0 ? c.i - P.Lx : -1, c.yi + 1 < P.Ly ? c.i + P.Lx : -1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (nb[q] < 0) continue;
      const float4 sq = s32[nb[q]];
      h0 += sq.x;
      h1 += sq.y;
      h2 += sq.z;
    }
    const float bj = P.bJ_f;
    tex = -bj * ((nx - ax) * h0 + (ny - ay) * h1 + (nz - az) * h2);
    bex = 0x1p-14f * fabsf(bj);
  }
  const float lo = logf(pz_o), ln = logf(pz_n);
  const float scale = (float)((sc_n - sc_o) * kScale32) * 0.693147182f;
  const float lu = logf((float)c.u);
  const float bdv = beta * (sum + comp);
  const float mu = lu + ((bdv + tex) + ((lo - ln) + scale));
  const float B = 2.0f * (2.0f * c0s * 1.001f + (float)(n + 2) * 0x1p-23f * beta * sum_abs +
                          lin * 1.001f + n * (0x1p-19f + 0x1p-22f) +
                          0x1p-21f * (fabsf(lo) + fabsf(ln)) + 0x1p-20f * fabsf(lu) + 0x1p-23f +
                          bex + 0x1p-21f * (fabsf(scale) + fabsf(tex) + fabsf(bdv) + fabsf(mu)));
  if (mu < -B) return 1;
  if (mu > B) return 0;
  return 2;
}

// Proposal of site i at MC step t (Philox tag PROPOSE, counter (i, t, a)); false if all 64
// attempts were rejected.
// The square root and the spin are computed once, after the attempts (whose count differs
// between the lanes of a warp).
__device__ __forceinline__ bool propose(const DevParams& P, SiteCtx& c, uint64_t step) {
  double a1 = 0.0, a2 = 0.0, s = 0.0;
  uint64_t wu = 0;
  bool ok = false;
  for (uint64_t a = 0; a < 64 && !ok; ++a) {
    const W4 w = philox((uint64_t)c.i, step, a, kTagPropose, P.key0, P.key1);
    ok = marsaglia_point(w.w[0], w.w[1], a1, a2, s);
    wu = w.w[2];
  }
  if (!ok) return false;
  marsaglia_spin(a1, a2, s, c.Sn[0], c.Sn[1], c.Sn[2]);
  c.u = u53(wu);
  return true;
}

// Proposals are drawn for every site of a lattice by k_propose before the colour classes of a
// step run (they depend only on (seed, site, step)), one double4 {S'x, S'y, S'z, u} per site;
// u = -1 marks a site whose 64 attempts were all rejected (no move).
__device__ __forceinline__ bool take_proposal(SiteCtx& c, const double4_32a* __restrict__ prop) {
  const double4_32a q = prop[c.i];
  c.Sn[0] = q.x;
  c.Sn[1] = q.y;
  c.Sn[2] = q.z;
  c.u = q.w;
  return q.w >= 0.0;
}

__device__ __forceinline__ void load_site(const DevParams& P, SiteCtx& c, uint32_t i,
                                          const double* __restrict__ s) {
  c.i = i;
  c.yi = (int32_t)site_row(i, P);
  c.xi = (int32_t)(i - (uint32_t)c.yi * (uint32_t)P.Lx);
  c.S[0] = s[i];
  c.S[1] = s[P.N + i];
  c.S[2] = s[2 * P.N + i];
}

__device__ __forceinline__ void write_site(const DevParams& P, const SiteCtx& c, bool ok,
                                           double* __restrict__ s, float4* __restrict__ s32,
                                           uint8_t* __restrict__ acc) {
  if (ok) {
    s[c.i] = c.Sn[0];
    s[P.N + c.i] = c.Sn[1];
    s[2 * P.N + c.i] = c.Sn[2];
    if (s32) s32[c.i] = make_float4((float)c.Sn[0], (float)c.Sn[1], (float)c.Sn[2], 0.f);
  }
  acc[c.i] = ok ? 1 : 0;
}

// Product over the warp of the lanes' p 2^(-600 sc) (p a positive normal double): mantissa m in
// [1, 2) and exponent e on every lane (the butterfly multiplies the same pairs on both lanes of
// a step, so all lanes end with the same bits).
__device__ __forceinline__ void warp_prod(double p, int sc, double& m, int& e) {
  const unsigned long long b = pos_bits(p);
  e = (int)(b >> 52) - 1023 - kScale64 * sc;
  m = __longlong_as_double((long long)((b & 0xFFFFFFFFFFFFFull) | 0x3FF0000000000000ull));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m *= __shfl_xor_sync(0xffffffffu, m, o);
    e += __shfl_xor_sync(0xffffffffu, e, o);
    const unsigned long long mb = pos_bits(m);
    if ((mb >> 52) > 1023u) {  // m in [2, 4): halve it exactly
      m = __longlong_as_double((long long)(mb - (1ull << 52)));
      ++e;
    }
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_min_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ dd warp_sum_dd(dd v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const dd w = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = dd_add(v, w);
  }
  return v;
}

// The FP64 decision of accept_fp64 with the pairs of the site spread over the 32 lanes of a
// warp (partial sums, products taken to logarithms per lane, then reduced).  Same bound, plus
// the per-lane logarithms.
__device__ int accept_fp64_warp(const DevParams& P, const SiteCtx& c,
                                const Sw64* __restrict__ sw,
                                const double* __restrict__ s,
                                const uint32_t* __restrict__ row_ptr,
                                const uint32_t* __restrict__ col, int lane) {
  double bdv = 0.0, pz_o = 1.0, pz_n = 1.0, c0s = 0.0;
  int sc_o = 0, sc_n = 0, n = 0, bad = 0, dmax = -2046;
  const uint32_t e1 = row_ptr[c.i + 1];
  for (uint32_t e = row_ptr[c.i] + lane; e < e1; e += 32) {
    const uint32_t cj = col[e];
    if (cj & kExchOnly) continue;
    const uint32_t j = cj;
    const uint32_t yj = site_row(j, P);
    const int32_t dx = (int32_t)(j - yj * (uint32_t)P.Lx) - c.xi;
    const int32_t dy = (int32_t)yj - c.yi;
    const Sw64& t = sw[(int64_t)(dx < 0 ? -dx : dx) + (int64_t)P.Lx * (dy < 0 ? -dy : dy)];
    const double fx = flip_if(t.ax, dx < 0), fy = flip_if(t.ay, dy < 0);
    const double ax3 = flip_if(t.a3x, dx < 0), ay3 = flip_if(t.a3y, dy < 0);
    const double bx = s[j], by = s[P.N + j], bz = s[2 * P.N + j];
    const double tp = bx * ax3 + by * ay3;
    const double gx = t.a1 * bx - tp * fx;
    const double gy = t.a1 * by - tp * fy;
    const double gz = t.a1 * bz;
    const double xn = fma(c.Sn[0], gx, fma(c.Sn[1], gy, fma(c.Sn[2], gz, -t.bvm)));
    const double xo = fma(c.S[0], gx, fma(c.S[1], gy, fma(c.S[2], gz, -t.bvm)));
    if (!neg_strict(xn) || !neg_strict(xo)) {
      bad = 1;
      continue;
    }
    const double zn = neg_expm1_np6(xn), zo = neg_expm1_np6(xo);
    pz_n *= zn;
    pz_o *= zo;
    if (!renorm600(pz_n, sc_n) || !renorm600(pz_o, sc_o)) bad = 1;
    bdv += xn - xo;
    dmax = max(dmax, exp_field(t.c0) - min(exp_field(zn), exp_field(zo)));
    c0s += t.c0;
    ++n;
  }
  // per lane: log of its products, with the renormalisation folded in
  const double lo = log_np(pz_o) - (double)(sc_o * kScale64) * P.ln2_hi;
  const double ln = log_np(pz_n) - (double)(sc_n * kScale64) * P.ln2_hi;
  const double lsum = warp_sum_d(lo - ln);
  const double labs = warp_sum_d(fabs(lo) + fabs(ln));
  bdv = warp_sum_d(bdv);
  c0s = warp_sum_d(c0s);
  dmax = __reduce_max_sync(0xffffffffu, dmax);
  n = __reduce_add_sync(0xffffffffu, n);
  bad = __reduce_or_sync(0xffffffffu, bad);
  if (bad) return 2;
  if (n > 0 && dmax + 2 + (32 - __clz(n)) > -10) return 2;
  // n 2^(dmax + 2), the power of two from its bits (dmax + 2 <= -10 here; below -1022: 0)
  const double lin = n > 0 && dmax + 2 >= -1022
                         ? (double)n * __longlong_as_double((long long)(dmax + 2 + 1023) << 52)
                         : 0.0;
  double tex = 0.0, bex = 0.0;
  if (P.J != 0.0) {
    double h0 = 0.0, h1 = 0.0, h2 = 0.0;
    const int64_t nb[4] = {c.xi > 0 ? c.i - 1 : -1, c.xi + 1 < P.Lx ? c.i + 1 : -1,
                           c.yi > 0 ? c.i - P.Lx : -1, c.yi + 1 < P.Ly ? c.i + P.Lx : -1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (nb[q] < 0) continue;
      h0 += s[nb[q]];
      h1 += s[P.N + nb[q]];
      h2 += s[2 * P.N + nb[q]];
    }
    const double dot = (c.Sn[0] - c.S[0]) * h0 + (c.Sn[1] - c.S[1]) * h1 + (c.Sn[2] - c.S[2]) * h2;
    tex = -(P.beta * P.J) * dot;
    bex = 0x1p-44 * fabs(P.beta * P.J);
  }
  const double lu = log_np(c.u);
  const double mu = lu + ((bdv + tex) + lsum);
  const double B = 2.0 * ((double)(n + 4) * c0s + 2.0 * lin + n * (4.0 * kExpm1RelErr6 + 0x1p-51) +
                          kLogRelErr * (labs + fabs(lu)) + 0x1p-49 * labs + bex +
                          0x1p-51 * (fabs(tex) + fabs(bdv) + fabs(mu)));
  if (mu < -B) return 1;
  if (mu > B) return 0;
  return 2;
}

// accept_fp64_warp with the pair cache (see accept_fp64_cached); every lane writes the
// proposed-spin terms of its pairs.
__device__ int accept_fp64_warp_cached(const DevParams& P, const SiteCtx& c,
                                       const Sw64* __restrict__ sw,
                                       const double* __restrict__ s,
                                       const uint32_t* __restrict__ row_ptr,
                                       const uint32_t* __restrict__ col, const PairCache& pc,
                                       uint32_t ui, int lane) {
  double bdv = 0.0, pz_o = 1.0, pz_n = 1.0, c0s = 0.0;
  int sc_o = 0, sc_n = 0, n = 0, bad = 0, dmax = -2046;
  const uint32_t e1 = row_ptr[c.i + 1];
  for (uint32_t e = row_ptr[c.i] + lane; e < e1; e += 32) {
    const uint32_t cj = col[e];
    if (cj & kExchOnly) continue;
    const uint32_t j = cj;
    const uint32_t h = pc.hid[e];
    const uint32_t uj = pc.upd[j];
    const uint32_t yj = site_row(j, P);
    const int32_t dx = (int32_t)(j - yj * (uint32_t)P.Lx) - c.xi;
    const int32_t dy = (int32_t)yj - c.yi;
    const Sw64& t = sw[(int64_t)(dx < 0 ? -dx : dx) + (int64_t)P.Lx * (dy < 0 ? -dy : dy)];
    const double fx = flip_if(t.ax, dx < 0), fy = flip_if(t.ay, dy < 0);
    const double ax3 = flip_if(t.a3x, dx < 0), ay3 = flip_if(t.a3y, dy < 0);
    const double bx = s[j], by = s[P.N + j], bz = s[2 * P.N + j];
    double2* rec = reinterpret_cast<double2*>(&pc.keep[h]);
    const uint32_t hf = ((ui ^ uj) >> 2) & 1u;
    const double2 kv = rec[hf];
    const double zo = kv.x, xo = kv.y;
    const double ns = c.Sn[0] * bx + c.Sn[1] * by + c.Sn[2] * bz;
    const double tp = bx * ax3 + by * ay3;
    const double nd = c.Sn[0] * fx + c.Sn[1] * fy;
    const double xn = fma(t.a1, ns, fma(-tp, nd, -t.bvm));
    const bool okn = neg_strict(xn);
    const double zn = okn ? neg_expm1_np6(xn) : -1.0;
    if ((uj & 3u) == 0u || pc.carry) rec[hf ^ 1u] = make_double2(zn, xn);
    if (!okn || !neg_strict(xo) || !(pos_bits(zo) - 1ull < 0x7FEFFFFFFFFFFFFFull)) {
      bad = 1;
      continue;
    }
    pz_n *= zn;
    pz_o *= zo;
    if (!renorm600(pz_n, sc_n) || !renorm600(pz_o, sc_o)) bad = 1;
    bdv += xn - xo;
    dmax = max(dmax, exp_field(t.c0) - min(exp_field(zn), exp_field(zo)));
    c0s += t.c0;
    ++n;
  }
  bdv = warp_sum_d(bdv);
  c0s = warp_sum_d(c0s);
  dmax = __reduce_max_sync(0xffffffffu, dmax);
  n = __reduce_add_sync(0xffffffffu, n);
  bad = __reduce_or_sync(0xffffffffu, bad);
  if (bad) return 2;
  if (n > 0 && dmax + 2 + (32 - __clz(n)) > -10) return 2;
  double mo, mn;
  int eo, en;
  warp_prod(pz_o, sc_o, mo, eo);
  warp_prod(pz_n, sc_n, mn, en);
  const double lin = n > 0 && dmax + 2 >= -1022
                         ? (double)n * __longlong_as_double((long long)(dmax + 2 + 1023) << 52)
                         : 0.0;
  double tex = 0.0, bex = 0.0;
  if (P.J != 0.0) {
    double h0 = 0.0, h1 = 0.0, h2 = 0.0;
    const int64_t nb[4] = {c.xi > 0 ? c.i - 1 : -1, c.xi + 1 < P.Lx ? c.i + 1 : -1,
                           c.yi > 0 ? c.i - P.Lx : -1, c.yi + 1 < P.Ly ? c.i + P.Lx : -1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (nb[q] < 0) continue;
      h0 += s[nb[q]];
      h1 += s[P.N + nb[q]];
      h2 += s[2 * P.N + nb[q]];
    }
    const double dot = (c.Sn[0] - c.S[0]) * h0 + (c.Sn[1] - c.S[1]) * h1 + (c.Sn[2] - c.S[2]) * h2;
    tex = -(P.beta * P.J) * dot;
    bex = 0x1p-44 * fabs(P.beta * P.J);
  }
  // the product form of accept_fp64_cached on the warp's products mo 2^eo and mn 2^en (the
  // butterfly's ten products add 2^-49 to the 2^-31 term)
  const double A = bdv + tex;
  const double t = fma(A, kExpInvLn2, 0x1.8p52);
  const double kd = t - 0x1.8p52;
  const int k = __double2loint(t);
  if (k > (1 << 20) || k < -(1 << 20)) return 2;
  const double r = fma(-kd, kExpLn2, A);
  const double er = fma(r, expm1_poly6(r), 1.0);
  const double X = (c.u * mo) * er;
  const double delta = 2.0 * ((double)(n + 4) * c0s + 2.0 * lin +
                              n * (4.0 * kExpm1RelErr6 + 0x1p-51) + bex +
                              0x1p-51 * (fabs(tex) + fabs(bdv)) + 0x1p-31);
  if (!(delta < 0.25)) return 2;
  const int eX = exp_field(X);
  if (eX == 0) return 1;  // u = 0
  const int dE = eX - 1023 + k + eo - en;  // mn in [1, 2)
  if (dE >= 2) return 0;
  if (dE <= -2) return 1;
  const double Xs = __longlong_as_double(__double_as_longlong(X) + ((long long)(dE + 1023 - eX) << 52));
  const double D = Xs - mn;
  const long long oD = ord_bits(D), ol = ord_bits(delta * mn);
  if (oD < -ol - 1) return 1;
  if (oD > ol) return 0;
  return 2;
}

// The same comparison in double-double, pairs spread over the lanes.
__device__ bool accept_dd_warp(const DevParams& P, const SiteCtx& c,
                               const double* __restrict__ s,
                               const uint32_t* __restrict__ row_ptr,
                               const uint32_t* __restrict__ col, int lane) {
  const dd ln2 = {P.ln2_hi, P.ln2_lo};
  dd sum = dd_from(0.0);
  int inf = 0;
  const uint32_t e1 = row_ptr[c.i + 1];
  for (uint32_t e = row_ptr[c.i] + lane; e < e1; e += 32) {
    const uint32_t cj = col[e];
    if (cj & kExchOnly) continue;
    const uint32_t j = cj;
    const uint32_t yj = site_row(j, P);
    const int32_t dx = (int32_t)(j - yj * (uint32_t)P.Lx) - c.xi;
    const int32_t dy = (int32_t)yj - c.yi;
    const int64_t r2 = (int64_t)dx * dx + (int64_t)dy * dy;
    const double cc = coupling_c(r2);
    const dd Vm = dd_vmax(P.D, hazard_A(r2));
    const double Sj[3] = {s[j], s[P.N + j], s[2 * P.N + j]};
    const dd Vn = dd_pair_V(P.D, cc, (double)r2, c.Sn, Sj, (double)dx, (double)dy);
    const dd Vo = dd_pair_V(P.D, cc, (double)r2, c.S, Sj, (double)dx, (double)dy);
    const dd xn = dd_mul_d(dd_sub(Vn, Vm), P.beta);
    const dd xo = dd_mul_d(dd_sub(Vo, Vm), P.beta);
    if (!(xn.hi < 0.0)) {  // Vbar(S') = +inf
      inf = 1;
      continue;
    }
    sum = dd_add(sum, dd_mul_d(dd_sub(Vn, Vo), P.beta));
    sum = dd_sub(sum, dd_log1mexp(xn, ln2));
    sum = dd_add(sum, dd_log1mexp(xo, ln2));
  }
  sum = warp_sum_dd(sum);
  if (__reduce_or_sync(0xffffffffu, inf)) return false;
  if (P.J != 0.0) {
    dd h[3] = {dd_from(0.0), dd_from(0.0), dd_from(0.0)};
    const int64_t nb[4] = {c.xi > 0 ? c.i - 1 : -1, c.xi + 1 < P.Lx ? c.i + 1 : -1,
                           c.yi > 0 ? c.i - P.Lx : -1, c.yi + 1 < P.Ly ? c.i + P.Lx : -1};
    for (int q = 0; q < 4; ++q) {
      if (nb[q] < 0) continue;
      for (int a = 0; a < 3; ++a) h[a] = dd_add(h[a], dd_from(s[a * P.N + nb[q]]));
    }
    dd dot = dd_from(0.0);
    for (int a = 0; a < 3; ++a) dot = dd_add(dot, dd_mul(two_sum(c.Sn[a], -c.S[a]), h[a]));
    sum = dd_sub(sum, dd_mul(dot, two_prod(P.beta, P.J)));
  }
  const dd lu = dd_log(dd_from(c.u), ln2);
  return dd_lt(dd_add(lu, sum), dd_from(0.0));
}

}  // namespace
}  // namespace sco
