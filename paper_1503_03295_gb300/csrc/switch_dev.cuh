// switch_dev.cuh -- per-site body of step (A) of Sec. 2.1 (potential switching), shared by
// the single-lattice and the batched switch kernels.
//
// Every pair {i, i+d} survives (V -> Vbar) with probability 1 - P_ij, P_ij of Eq. (2),
// independently.  Site i visits its half-plane list by bound thinning: element m becomes a
// candidate with probability q_m = 1 - exp(-2 beta Vmax_m) (a Poisson process of rate
// beta D A_m 2^-58 per element, walked over the prefix W), and a candidate survives with
// probability (1 - P_ij) / q_m.  The draws come from Philox tag SWITCH, counter
// (i, epoch, n/2), draw n using words 2(n%2) (exponential) and 2(n%2)+1 (survival).
//
// Every decision is an exact comparison of reals built from FP64 inputs.  It is taken in
// FP64 (or FP32 in the FP32-guarded form) together with a bound on the rounding error; a
// margin inside the bound sends the decision to double-double arithmetic.
#pragma once

#include <cstdint>

#include "sco_internal.h"

namespace sco {
namespace {

constexpr int kNear = 2048;  // head of the sorted list kept in shared memory (r <~ 25)
constexpr int kStatusCapacity = 7;

__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, 0, code); }

// The sorted half-plane list as a walk reads it: displacements d, the hazard prefix W and (FP64
// search) the decay bits E of Table::Ebits, the first nnear displacements in shared memory with
// the first nw entries of W (nw = nnear, or 0 when the shared array holds E instead).
struct NearTable {
  const uint64_t* sW;
  const uint32_t* sD;
  const uint64_t* W;
  const uint32_t* disp;
  int64_t nnear, K, nw;
  const uint64_t* sE = nullptr;  // first nnear decay bits (FP64 search), or nullptr
  const uint64_t* E = nullptr;   // all K decay bits, or nullptr: search W with a logarithm
  uint64_t elast = 0;            // E[K - 1]
  __device__ __forceinline__ uint64_t w(int64_t k) const { return k < nw ? sW[k] : __ldg(&W[k]); }
  __device__ __forceinline__ uint32_t d(int64_t k) const {
    return k < nnear ? sD[k] : __ldg(&disp[k]);
  }
  __device__ __forceinline__ uint64_t e(int64_t k) const {
    return k < nnear ? sE[k] : __ldg(&E[k]);
  }
  // first k in [lo, K) with W[k] >= target, K if none
  __device__ __forceinline__ int64_t lower_bound(int64_t lo, uint64_t target) const {
    if (lo < nw) {
      if (sW[nw - 1] >= target) {
        int64_t a = lo, b = nw - 1;
        while (a < b) {
          const int64_t mid = (a + b) >> 1;
          if (sW[mid] >= target) b = mid; else a = mid + 1;
        }
        return a;
      }
      lo = nw;
    }
    int64_t a = lo, b = K;
    while (a < b) {
      const int64_t mid = (a + b) >> 1;
      if (__ldg(&W[mid]) >= target) b = mid; else a = mid + 1;
    }
    return a;
  }
  // first k in [lo, K) with E[k] <= target (E is non-increasing), K if none
  __device__ __forceinline__ int64_t lower_bound_e(int64_t lo, uint64_t target) const {
    if (lo < nnear) {
      if (sE[nnear - 1] <= target) {
        int64_t a = lo, b = nnear - 1;
        while (a < b) {
          const int64_t mid = (a + b) >> 1;
          if (sE[mid] <= target) b = mid; else a = mid + 1;
        }
        return a;
      }
      lo = nnear;
    }
    int64_t a = lo, b = K;
    while (a < b) {
      const int64_t mid = (a + b) >> 1;
      if (__ldg(&E[mid]) <= target) b = mid; else a = mid + 1;
    }
    return a;
  }
};

// Exact re-evaluation of the next candidate: min { k > s : beta D 2^-58 (W_k - W_s) >= -ln u+ }.
// The table view comes by value (its address would put the caller's copy in local memory).
__device__ __noinline__ int64_t next_candidate_dd(const DevParams& P, const NearTable T,
                                                  int64_t s, uint64_t Ws, double up) {
  const dd ln2 = {P.ln2_hi, P.ln2_lo};
  const dd E = dd_neg(dd_log(dd_from(up), ln2));
  const dd tau = dd_ldexp(dd_div(E, two_prod(P.beta, P.D)), 58);
  int64_t a = s + 1, b = T.K;
  while (a < b) {
    const int64_t mid = (a + b) >> 1;
    if (!dd_lt(dd_from_u64(T.w(mid) - Ws), tau)) b = mid; else a = mid + 1;
  }
  return a;
}

__device__ __forceinline__ int64_t next_candidate(const DevParams& P, const NearTable& T,
                                                  int64_t s, uint64_t Ws, uint64_t Wtot,
                                                  uint64_t wE, unsigned& ghits);

// ceil(x) as an integer for finite x >= 0 (saturating at 2^64 - 1), from the bits of x with
// integer operations only (64-bit conversions would run on the FP64 pipe).
__device__ __forceinline__ uint64_t ceil_u64d(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  if (b == 0ull || (b >> 63)) return 0ull;
  const int ex = (int)((b >> 52) & 0x7FFu) - 1075;  // x = mant * 2^ex
  const uint64_t mant = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  if (ex >= 0) return ex >= 11 ? ~0ull : mant << ex;
  if (ex <= -54) return 1ull;  // 0 < x < 1
  const uint64_t q = mant >> (-ex);
  return q + ((q << (-ex)) != mant ? 1ull : 0ull);
}

__device__ __forceinline__ uint64_t ceil_u64(float x) {
  const uint32_t b = __float_as_uint(x);
  if (b == 0u || (b >> 31)) return 0ull;
  const int ex = (int)((b >> 23) & 0xFFu) - 150;  // x = mant * 2^ex
  const uint64_t mant = (uint64_t)((b & 0x7FFFFFu) | 0x800000u);
  if (ex >= 0) return ex >= 40 ? ~0ull : mant << ex;
  if (ex <= -25) return 1ull;  // 0 < x < 1
  const uint64_t q = mant >> (-ex);
  return q + ((q << (-ex)) != mant ? 1ull : 0ull);
}

// tau = -ln(u+) / (beta D 2^-58) carries < 2^-48 relative error (log_np within kLogRelErr =
// 2^-49, fl(beta D), fl(2^58 / bD), one product); the candidate is certain when
// W_k - W_s >= tau (1 + 2^-46) and
// W_(k-1) - W_s < tau (1 - 2^-46), compared as integers (ceil of the bounds).
__device__ __forceinline__ int64_t next_candidate(const DevParams& P, const NearTable& T,
                                                  int64_t s, uint64_t Ws, uint64_t Wtot,
                                                  uint64_t wE, unsigned& ghits) {
  if (s >= T.K - 1 || !P.switching) return T.K;
  const double up = u53pos(wE);
  const double tau = -log_np(up) * P.inv_bD58;
  const uint64_t rem = Wtot - Ws;
  const uint64_t thr = ceil_u64d(tau);
  int64_t k = T.K;
  if (thr <= rem) k = T.lower_bound(s + 1, Ws + thr);
  // thr = ceil(tau): ceil(tau (1 + 2^-46)) <= thr + floor(thr 2^-46) + 1 = hi and
  // tau (1 - 2^-46) >= (thr - 1)(1 - 2^-46) >= thr - floor(thr 2^-46) - 2 = lo (saturating),
  // in integers: no FP64 instruction
  const uint64_t m46 = thr >> 46;
  const uint64_t hi = thr + m46 + 1 < thr ? ~0ull : thr + m46 + 1;  // >= hi: surely a candidate
  const uint64_t lo = thr > m46 + 2 ? thr - m46 - 2 : 0ull;         // < lo: surely not
  bool certain = true;
  if (k < T.K && T.w(k) - Ws < hi) certain = false;
  if (k - 1 > s && T.w(k - 1) - Ws >= lo) certain = false;
  if (certain) return k;
  ++ghits;
  return next_candidate_dd(P, T, s, Ws, up);
}

// Bits of 1.0: the decay value before the first element (W = 0).
constexpr uint64_t kDecayStart = 0x3FF0000000000000ull;
// Targets below 2^-990 take the exact search (the decay table's values there are not normal).
constexpr uint64_t kDecayMinBits = 0x0210000000000000ull;

// FP64 candidate search without a logarithm.  With E*_m = exp(-beta D 2^-58 W_m) the next
// candidate min { k > s : beta D 2^-58 (W_k - W_s) >= -ln u+ } is min { k > s : E*_k <= u+ E*_s }
// (exp is increasing), searched on the table's bits: E_m within 2^-52 of E*_m, the target
// fl(u+ E_s) within 2^-51.9 of u+ E*_s.  Positive doubles order as their bit images, and 16
// units in the last place are at least 2^-49 relative, more than the combined error, so the
// candidate is certain when E_k's bits lie at least 16 below the target's and E_(k-1)'s at least
// 16 above; otherwise (or for a target below 2^-990) the search with the logarithm decides.
// Es carries the bits of E at the walk's last candidate and is advanced to the new one.
__device__ __forceinline__ int64_t next_candidate_e(const DevParams& P, const NearTable& T,
                                                    int64_t s, uint64_t& Es, uint64_t Wtot,
                                                    uint64_t wE, unsigned& ghits) {
  if (s >= T.K - 1 || !P.switching) return T.K;
  const uint64_t tb = (uint64_t)__double_as_longlong(u53pos(wE) * __longlong_as_double(Es));
  if (tb >= kDecayMinBits) {
    if (T.elast >= tb + 16ull) return T.K;  // surely no candidate left: the walk ends
    const int64_t k = T.lower_bound_e(s + 1, tb);
    const uint64_t ek = k < T.K ? T.e(k) : 0ull;
    bool certain = true;
    if (k < T.K && ek + 16ull > tb) certain = false;
    if (k - 1 > s && T.e(k - 1) < tb + 16ull) certain = false;
    if (certain) {
      Es = ek;
      return k;
    }
  }
  const int64_t k = next_candidate(P, T, s, s >= 0 ? T.w(s) : 0ull, Wtot, wE, ghits);
  if (k < T.K) Es = T.e(k);
  return k;
}

// FP32 screen of the candidate search.  E = -ln u+ is taken as -log1pf(-(1 - u+)) above 1/2
// (1 - u+ is an exact integer times 2^-53) and -logf(u+) below, so its relative error stays
// below 2^-20.5 (one input rounding, 4 ulp of the function); tau = E fl32(2^58 / bD) adds
// two roundings.  Margins inside 2^-18 fall through to the FP64 search.  All comparisons
// with the uint64 prefix W are made in integers.
__device__ __forceinline__ int64_t next_candidate_fp32(const DevParams& P, const NearTable& T,
                                                       int64_t s, uint64_t Ws, uint64_t Wtot,
                                                       uint64_t wE, unsigned& g32,
                                                       unsigned& ghits) {
  if (s >= T.K - 1 || !P.switching) return T.K;
  const uint64_t m53 = wE >> 11;  // u+ = (m53 + 1) 2^-53
  float E;
  if (m53 >= (1ull << 52)) {
    const uint64_t dm = (1ull << 53) - 1ull - m53;  // < 2^52
    const float d = __uint2float_rn((uint32_t)(dm >> 20)) * 0x1p-33f +
                    __uint2float_rn((uint32_t)(dm & 0xFFFFFu)) * 0x1p-53f;
    E = -log1pf(-d);
  } else {
    const uint64_t um = m53 + 1ull;  // <= 2^52
    const float u = __uint2float_rn((uint32_t)(um >> 20)) * 0x1p-33f +
                    __uint2float_rn((uint32_t)(um & 0xFFFFFu)) * 0x1p-53f;
    E = -logf(u);
  }
  const float tau = E * P.inv_bD58_f;
  const uint64_t rem = Wtot - Ws;
  const uint64_t thr = ceil_u64(tau);
  int64_t k = T.K;
  if (thr <= rem) k = T.lower_bound(s + 1, Ws + thr);
  // margins 2^-18 around tau from thr = ceil(tau), in integers (conservative, as in the FP64
  // search): ceil(tau (1 + 2^-18)) <= thr + floor(thr 2^-18) + 1 = hi, and
  // tau (1 - 2^-18) >= thr - floor(thr 2^-18) - 2 = lo (saturating)
  const uint64_t m18 = thr >> 18;
  const uint64_t hi = thr + m18 + 1 < thr ? ~0ull : thr + m18 + 1;  // >= hi: surely a candidate
  const uint64_t lo = thr > m18 + 2 ? thr - m18 - 2 : 0ull;         // < lo: surely not
  bool certain = tau < 0x1p62f;
  if (k < T.K && T.w(k) - Ws < hi) certain = false;
  if (k - 1 > s && T.w(k - 1) - Ws >= lo) certain = false;
  if (certain) return k;
  ++g32;
  return next_candidate(P, T, s, Ws, Wtot, wE, ghits);
}

// Exact survival test u q < 1 - P_ij in double-double.  The spins come by value, so that the
// callers' spin copies stay in registers (an address passed to a function that is not inlined
// would put them in local memory on the fast path too).
__device__ __noinline__ bool survives_dd(const DevParams& P, double si0, double si1, double si2,
                                         double sj0, double sj1, double sj2, int32_t dx,
                                         int32_t dy, uint64_t A, double u1) {
  const double Si[3] = {si0, si1, si2}, Sj[3] = {sj0, sj1, sj2};
  const dd ln2 = {P.ln2_hi, P.ln2_lo};
  const int64_t r2 = (int64_t)dx * dx + (int64_t)dy * dy;
  const dd V = dd_pair_V(P.D, coupling_c(r2), (double)r2, Si, Sj, (double)dx, (double)dy);
  const dd Vm = dd_vmax(P.D, A);
  const dd b = dd_mul_d(dd_sub(V, Vm), P.beta);
  const dd a = dd_mul_d(Vm, 2.0 * P.beta);
  const dd pr = dd_neg(dd_expm1(b, ln2));
  const dd q = dd_neg(dd_expm1(dd_neg(a), ln2));
  return dd_lt(dd_mul_d(q, u1), pr);
}

// 1 - P_ij = -expm1(beta (V - Vmax)) of the pair (S_i at i, S_j at i + (dx, dy)) in FP64 from the
// beta-scaled pair table t: x = a1 (S_i.S_j) - (S_i.a3 d)(S_j.d) - bvm, |x error| <= c0 +
// 2^-52 |x| (c0 covers the roundings), then expm1_np6 (relative error kExpm1RelErr6).
// x itself is returned in *x.
__device__ __forceinline__ double pair_keep64(const Sw64& t, const double* Si, const double* Sj,
                                              int32_t dx, int32_t dy, double* x) {
  const double fx = flip_if(t.ax, dx < 0), fy = flip_if(t.ay, dy < 0);
  const double ax3 = flip_if(t.a3x, dx < 0), ay3 = flip_if(t.a3y, dy < 0);
  const double ss = Si[0] * Sj[0] + Si[1] * Sj[1] + Si[2] * Sj[2];
  const double pa = Si[0] * ax3 + Si[1] * ay3;
  const double pb = Sj[0] * fx + Sj[1] * fy;
  const double b = fma(t.a1, ss, fma(-pa, pb, -t.bvm));  // c0 covers these two roundings
  *x = b;
  return neg_expm1_np6(b);
}

// The integer hazard A_k of list element k (only the double-double tests need it).
__device__ __forceinline__ uint64_t hazard_of(const NearTable& T, int64_t k) {
  return T.w(k) - (k > 0 ? T.w(k - 1) : 0ull);
}

// Bits of 2^-990: below it the survival test's relative margin is not formed from the exponent.
constexpr long long kRelMinBits = 0x0210000000000000ll;

// FP64 survival test u q < 1 - P_ij: x = beta (V - Vmax) from the beta-scaled pair table
// (t, the sweep's Sw64 entry), 1 - P = -expm1_np6(x).  The error of mu = (1 - P) - u q is below
// t.bsw / 4 (|dx| <= c0, q within 2^-50, two roundings; precomputed) plus 2^-31 (1 - P)
// (expm1_np6); the test is certain when |mu| exceeds twice the larger of the two doubled parts,
// i.e. both t.bsw and 2^-28 (1 - P), compared as ordered bit images (2^-28 (1 - P) by the
// exponent field, for 1 - P >= 2^-990).  u is exact.  `keep` receives the FP64 value of 1 - P
// (within its error bound whatever the decision).
__device__ __forceinline__ bool survives_fp64(const DevParams& P, const Sw64& t, double q,
                                              const double* Si, const double* Sj, int32_t dx,
                                              int32_t dy, const NearTable& T, int64_t k,
                                              double u1, unsigned& ghits, double& keep,
                                              double& xk) {
  const double pr = pair_keep64(t, Si, Sj, dx, dy, &xk);
  keep = pr;
  const double mu = pr - u1 * q;
  // mu > lim, mu < -lim on ordered bit images (lim > 0: ord(-lim) = -ord(lim) - 1)
  const long long pb = __double_as_longlong(pr);
  const long long ob = max(ord_bits(t.bsw), pb - (28ll << 52)), om = ord_bits(mu);
  if (pb >= kRelMinBits && om > ob) return true;
  if (pb >= kRelMinBits && om < -ob - 1) return false;
  ++ghits;
  return survives_dd(P, Si[0], Si[1], Si[2], Sj[0], Sj[1], Sj[2], dx, dy, hazard_of(T, k), u1);
}

// FP32 screen of the same test (FP32-guarded form): spins from the FP32 shadow
// (|dS| <= 2^-24 per component), table constants rounded to FP32, expm1f within 4 ulp.
// Falls through to the FP64 test (and from there to double-double) inside the bound; only
// then are the FP64 spins of i and j read from the SoA array s.
__device__ __forceinline__ bool survives_fp32(const DevParams& P, float4 t32,
                                              const Sw64* __restrict__ sw, double q64,
                                              const float* Si32, const float* Sj32,
                                              const double* __restrict__ s, int64_t i, int64_t j,
                                              int32_t dx, int32_t dy, const NearTable& T,
                                              int64_t k, uint64_t wU, unsigned& g32,
                                              unsigned& ghits) {
  const float fr2 = (float)(dx * dx + dy * dy), fx = (float)dx, fy = (float)dy;
  // u truncated to 24 bits: 0 <= u - u24 < 2^-24, inside the 2^-19 q term of the bound
  const float u24 = __uint2float_rn((uint32_t)(wU >> 40)) * 0x1p-24f;
  const float ss = Si32[0] * Sj32[0] + Si32[1] * Sj32[1] + Si32[2] * Sj32[2];
  const float pa = Si32[0] * fx + Si32[1] * fy;
  const float pb = Sj32[0] * fx + Sj32[1] * fy;
  const float V = t32.x * (fr2 * ss - 3.0f * (pa * pb));
  const float beta = P.beta_f;
  const float b = beta * (V - t32.y);
  const float pr = -expm1f(b);
  const float q = t32.w;  // fl32 of the FP64 q: 2^-24 on top of its 4 ulp
  const float mu = pr - u24 * q;
  // |dV| <= 2^-17 Dc r^2 (shadow spins, FP32 products, constant rounding); beta and the
  // constants carry 2^-24 each; expm1f 4 ulp; generous factor 2.
  const float dV = 0x1p-17f * t32.x * fr2;
  const float B = 2.0f * (beta * (dV + 0x1p-22f * t32.y) + 0x1p-21f * fabsf(b) +
                          0x1p-19f * (fabsf(pr) + q) + 0x1p-21f * t32.z);
  if (mu > B) return true;
  if (mu < -B) return false;
  ++g32;
  const int64_t tix = (int64_t)(dx < 0 ? -dx : dx) + (int64_t)P.Lx * (dy < 0 ? -dy : dy);
  const double Si[3] = {s[i], s[P.N + i], s[2 * P.N + i]};
  const double Sj[3] = {s[j], s[P.N + j], s[2 * P.N + j]};
  double keep, xk;
  return survives_fp64(P, sw[tix], q64, Si, Sj, dx, dy, T, k, u53(wU), ghits, keep, xk);
}

// Where a site writes its upper neighbours: kSlotCap slots of its own (row `id` of hslot), then
// an overflow list shared by all sites (entry: site id, j | flag).  indeg counts lower
// neighbours per (local) site.  keep / keep_ovf (optional, FP64 form): the FP64 values of
// 1 - P_ij and of x = beta (V - Vmax) of each surviving dipolar pair, written to the first half
// of the pair-cache record at the same slot or overflow index (the cache that the FP64 sweep
// starts from).
struct SwitchOut {
  uint32_t* hslot;
  uint32_t* indeg;
  uint32_t* ovf;
  uint32_t ovf_cap;
  unsigned long long* ovf_n;
  int* status;
  double4_32a* keep = nullptr;
  double4_32a* keep_ovf = nullptr;
};

// One site's walk along its half-plane list: the candidate search of Sec. 2.1 with the state it
// carries from one candidate to the next, so that a thread can take the candidates one at a time
// (and take up another site when its list ends).
template <int PREC>
struct SiteWalk {
  uint32_t i;   // local site index (the Philox counter)
  uint32_t id;  // site id in the slots and the overflow list
  int32_t xi, yi;
  double Si[3];    // FP64 form
  float Si32[3];   // FP32-screened form
  int64_t sidx;    // last candidate (-1 before the first)
  uint64_t Ws;     // W at sidx, or with the decay table the bits of E at sidx
  uint32_t n;      // candidates drawn; Philox block n / 2, words 0-1 or 2-3
  W4 w;
  uint32_t n_out;
  bool nn0, nn1;
};

__device__ __forceinline__ void switch_emit(const SwitchOut& o, uint32_t id, uint32_t& n_out,
                                            uint32_t jv, double keep = 0.0, double xk = 0.0) {
  if (n_out < (uint32_t)kSlotCap) {
    o.hslot[(size_t)id * kSlotCap + n_out] = jv;
    if (o.keep)
      *reinterpret_cast<double2*>(&o.keep[(size_t)id * kSlotCap + n_out]) = make_double2(keep, xk);
  } else {
    const unsigned long long idx = atomicAdd(o.ovf_n, 1ull);
    if (idx < o.ovf_cap) {
      o.ovf[2 * idx] = id;
      o.ovf[2 * idx + 1] = jv;
      if (o.keep) *reinterpret_cast<double2*>(&o.keep_ovf[idx]) = make_double2(keep, xk);
    } else {
      set_status(o.status, kStatusCapacity);
    }
  }
  ++n_out;
  atomicAdd(&o.indeg[jv & kIndexMask], 1u);
}

template <int PREC>
__device__ __forceinline__ void walk_begin(const DevParams& P, const NearTable& T,
                                           const double* __restrict__ s,
                                           const float4* __restrict__ s32, uint32_t i,
                                           uint32_t id, SiteWalk<PREC>& a) {
  a.i = i;
  a.id = id;
  a.yi = (int32_t)site_row(i, P);
  a.xi = (int32_t)(i - (uint32_t)a.yi * (uint32_t)P.Lx);
  if (PREC == 0) {
    a.Si[0] = s[i];
    a.Si[1] = s[P.N + i];
    a.Si[2] = s[2 * P.N + i];
  } else {
    const float4 si = s32[i];
    a.Si32[0] = si.x;
    a.Si32[1] = si.y;
    a.Si32[2] = si.z;
  }
  a.sidx = -1;
  a.Ws = PREC == 0 && T.E ? kDecayStart : 0ull;
  a.n = 0;
  a.n_out = 0;
  a.nn0 = false;
  a.nn1 = false;
}

// Draws the next candidate of the walk and, if it lies on the lattice, tests its survival
// (emitting the pair if it survives).  Returns false once the list is exhausted.  sync_mask:
// the lanes of the warp that run this step together (0 when threads walk independently); they
// meet after the candidate search, whose loops run for different lengths (a far candidate
// searches the list in global memory), so that the FP64 survival test is issued once for all of
// them instead of once per group of lanes that left the search together.
template <int PREC>
__device__ __forceinline__ bool walk_step(const DevParams& P, const NearTable& T, uint64_t Wtot,
                                          const Sw64* __restrict__ sw,
                                          const double* __restrict__ xyq,
                                          const float4* __restrict__ xy32,
                                          const double* __restrict__ s,
                                          const float4* __restrict__ s32, uint32_t epoch,
                                          int32_t mnn0, int32_t mnn1, const SwitchOut& o,
                                          SiteWalk<PREC>& a, unsigned long long& n_dip,
                                          unsigned& ghits, unsigned& g32, unsigned sync_mask) {
  if ((a.n & 1u) == 0u)
    a.w = philox((uint64_t)a.i, epoch, (uint64_t)(a.n >> 1), kTagSwitch, P.key0, P.key1);
  const uint64_t wE = (a.n & 1u) ? a.w.w[2] : a.w.w[0];
  const uint64_t wU = (a.n & 1u) ? a.w.w[3] : a.w.w[1];
  ++a.n;
  const bool decay = PREC == 0 && T.E != nullptr;  // uniform
  const int64_t k = PREC == 1 ? next_candidate_fp32(P, T, a.sidx, a.Ws, Wtot, wE, g32, ghits)
                    : decay   ? next_candidate_e(P, T, a.sidx, a.Ws, Wtot, wE, ghits)
                              : next_candidate(P, T, a.sidx, a.Ws, Wtot, wE, ghits);
  if (sync_mask) __syncwarp(sync_mask);
  if (k >= P.K) return false;
  const uint32_t d = T.d(k);
  const int32_t dx = (int16_t)(d & 0xFFFFu), dy = (int32_t)(d >> 16);
  const int32_t xj = a.xi + dx, yj = a.yi + dy;
  if (xj >= 0 && xj < P.Lx && yj < P.Ly) {
    const int64_t j = xj + (int64_t)P.Lx * yj;
    const int64_t tix = (int64_t)(dx < 0 ? -dx : dx) + (int64_t)P.Lx * dy;
    bool surv;
    double keep = 0.0, xk = 0.0;
    if (PREC == 1) {
      const float4 sj = s32[j];
      const float Sj32[3] = {sj.x, sj.y, sj.z};
      surv = survives_fp32(P, __ldg(&xy32[tix]), sw, __ldg(&xyq[tix]), a.Si32, Sj32, s,
                           (int64_t)a.i, j, dx, dy, T, k, wU, g32, ghits);
    } else {
      const double Sj[3] = {s[j], s[P.N + j], s[2 * P.N + j]};
      surv = survives_fp64(P, sw[tix], __ldg(&xyq[tix]), a.Si, Sj, dx, dy, T, k, u53(wU), ghits,
                           keep, xk);
    }
    if (surv) {
      switch_emit(o, a.id, a.n_out, (uint32_t)j, keep, xk);
      ++n_dip;
      if (k == mnn0) a.nn0 = true;
      if (k == mnn1) a.nn1 = true;
    }
  }
  a.sidx = k;
  if (!decay) a.Ws = T.w(k);
  return true;
}

// Ends the walk: exchange bonds that the dipolar switch did not keep join the colouring graph.
// Returns the number of upper neighbours written (dipolar survivors plus exchange-only bonds).
template <int PREC>
__device__ __forceinline__ uint32_t walk_end(const DevParams& P, int32_t mnn0, int32_t mnn1,
                                             const SwitchOut& o, SiteWalk<PREC>& a) {
  if (P.J != 0.0) {
    if (mnn0 >= 0 && !a.nn0 && a.xi + 1 < P.Lx) switch_emit(o, a.id, a.n_out, (a.i + 1) | kExchOnly);
    if (mnn1 >= 0 && !a.nn1 && a.yi + 1 < P.Ly)
      switch_emit(o, a.id, a.n_out, (a.i + (uint32_t)P.Lx) | kExchOnly);
  }
  return a.n_out;
}

// Switches the half-plane pairs of site i (local index, slot id `id`) at this epoch in one go;
// returns the number of upper neighbours written.
template <int PREC>
__device__ __forceinline__ uint32_t switch_site(const DevParams& P, const NearTable& T,
                                                uint64_t Wtot, const Sw64* __restrict__ sw,
                                                const double* __restrict__ xyq,
                                                const float4* __restrict__ xy32,
                                                const double* __restrict__ s,
                                                const float4* __restrict__ s32, uint32_t epoch,
                                                int32_t mnn0, int32_t mnn1, uint32_t i,
                                                uint32_t id, const SwitchOut& o,
                                                unsigned long long& n_dip, unsigned& ghits,
                                                unsigned& g32) {
  SiteWalk<PREC> a;
  walk_begin<PREC>(P, T, s, s32, i, id, a);
  while (walk_step<PREC>(P, T, Wtot, sw, xyq, xy32, s, s32, epoch, mnn0, mnn1, o, a, n_dip,
                         ghits, g32, 0u)) {
  }
  return walk_end<PREC>(P, mnn0, mnn1, o, a);
}

// Compare-exchange on the neighbour index (the exchange flag travels with its entry).
__device__ __forceinline__ void row_ce(uint32_t& a, uint32_t& b) {
  const bool sw = (a & kIndexMask) > (b & kIndexMask);
  const uint32_t lo = sw ? b : a, hi = sw ? a : b;
  a = lo;
  b = hi;
}

// Sorts one CSR row by neighbour index; returns the number of dipolar entries of the row.
// Rows of at most 32 entries go through a bitonic network in registers (padded with
// 0xFFFFFFFF, whose index sorts after every site), longer ones through an insertion sort in
// place.  Neighbour indices inside a row are distinct, so the order is unique.
__device__ __forceinline__ unsigned sort_row(uint32_t* __restrict__ r, uint32_t n) {
  unsigned nd = 0;
  if (n <= 32) {
    uint32_t v[32];
#pragma unroll
    for (int a = 0; a < 32; ++a) v[a] = (uint32_t)a < n ? r[a] : 0xFFFFFFFFu;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
        for (int a = 0; a < 32; ++a) {
          const int l = a ^ j;
          if (l > a) {
            if ((a & k) == 0) row_ce(v[a], v[l]);
            else row_ce(v[l], v[a]);
          }
        }
      }
    }
#pragma unroll
    for (int a = 0; a < 32; ++a) {
      if ((uint32_t)a < n) {
        r[a] = v[a];
        nd += (v[a] & kExchOnly) ? 0u : 1u;
      }
    }
  } else {
    for (uint32_t a = 1; a < n; ++a) {
      const uint32_t x = r[a];
      uint32_t c = a;
      while (c > 0 && (r[c - 1] & kIndexMask) > (x & kIndexMask)) {
        r[c] = r[c - 1];
        --c;
      }
      r[c] = x;
    }
    for (uint32_t a = 0; a < n; ++a) nd += (r[a] & kExchOnly) ? 0u : 1u;
  }
  return nd;
}

}  // namespace
}  // namespace sco
