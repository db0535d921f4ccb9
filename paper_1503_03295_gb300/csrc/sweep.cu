// sweep.cu -- step (B) of Sec. 2.1 / step (3) of Fig. 1: Metropolis updates of all sites of
// one colour class at a time under the switched Hamiltonian H' of Eq. (4).
//
// Proposal for site i at MC step t: Philox tag PROPOSE, counter (i, t, a); attempt a uses
// words 0, 1 for Marsaglia's sphere point and word 2 of the successful attempt is the
// acceptance uniform u; 64 failed attempts keep the spin.  The move is accepted iff
// u < exp(-beta dE'), i.e. u == 0 or ln u + beta dE' < 0, with
//   beta dE' = sum_{surviving j} [beta V(S', S_j) - L(S') - beta V(S, S_j) + L(S)]
//              - beta J (S' - S) . sum_{nn j} S_j,
//   L = log(1 - exp(beta (V - Vmax)))   (so that beta Vbar = beta V - L, Eq. (3)).
// The decision is taken in FP64 (or FP32 in the FP32-guarded form) with a bound on the
// rounding error of the margin; margins inside the bound go to FP64 (from FP32) and then
// to double-double.  Sites of one colour share no pair, so they update independently.
#include <cstdint>

#include "sco_internal.h"

namespace sco {

namespace {

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

struct SiteCtx {
  int64_t i;
  int32_t xi, yi;
  double S[3], Sn[3];
  double u;
};

// Extended-precision evaluation of the same comparison.
__device__ __noinline__ bool accept_dd(const DevParams& P, const SiteCtx& c,
                                       const double* __restrict__ s,
                                       const uint32_t* __restrict__ row_ptr,
                                       const uint32_t* __restrict__ col) {
  const dd ln2 = {P.ln2_hi, P.ln2_lo};
  dd sum = dd_from(0.0);
  for (uint32_t e = row_ptr[c.i]; e < row_ptr[c.i + 1]; ++e) {
    const uint32_t cj = col[e];
    if (cj & kExchOnly) continue;
    const int64_t j = cj;
    const int32_t dx = (int32_t)(j % P.Lx) - c.xi, dy = (int32_t)(j / P.Lx) - c.yi;
    const int64_t r2 = (int64_t)dx * dx + (int64_t)dy * dy;
    const double cc = coupling_c(r2);
    const dd Vm = dd_vmax(P.D, hazard_A(r2));
    const double Sj[3] = {s[j], s[P.N + j], s[2 * P.N + j]};
    const dd Vn = dd_pair_V(P.D, cc, (double)r2, c.Sn, Sj, (double)dx, (double)dy);
    const dd Vo = dd_pair_V(P.D, cc, (double)r2, c.S, Sj, (double)dx, (double)dy);
    const dd xn = dd_mul_d(dd_sub(Vn, Vm), P.beta);
    const dd xo = dd_mul_d(dd_sub(Vo, Vm), P.beta);
    if (!(xn.hi < 0.0)) return false;  // Vbar(S') = +inf
    sum = dd_add(sum, dd_mul_d(dd_sub(Vn, Vo), P.beta));
    sum = dd_sub(sum, dd_log1mexp(xn, ln2));
    sum = dd_add(sum, dd_log1mexp(xo, ln2));
  }
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

// FP64 decision with its error bound (0: reject, 1: accept, 2: undecided).
__device__ __forceinline__ int accept_fp64(const DevParams& P, const SiteCtx& c,
                                           const double2* __restrict__ xy,
                                           const double* __restrict__ s,
                                           const uint32_t* __restrict__ row_ptr,
                                           const uint32_t* __restrict__ col) {
  double sum = 0.0, sumabs = 0.0, bnd = 0.0;
  int nterm = 0;
  const double beta = P.beta;
  for (uint32_t e = row_ptr[c.i]; e < row_ptr[c.i + 1]; ++e) {
    const uint32_t cj = col[e];
    if (cj & kExchOnly) continue;
    const int64_t j = cj;
    const int32_t dx = (int32_t)(j % P.Lx) - c.xi, dy = (int32_t)(j / P.Lx) - c.yi;
    const double2 t = __ldg(&xy[(int64_t)(dx < 0 ? -dx : dx) + (int64_t)P.Lx * (dy < 0 ? -dy : dy)]);
    const double r2 = (double)dx * dx + (double)dy * dy;
    const double bx = s[j], by = s[P.N + j], bz = s[2 * P.N + j];
    const double fx = (double)dx, fy = (double)dy;
    const double Vn = pair_V(t.x, r2, c.Sn[0], c.Sn[1], c.Sn[2], bx, by, bz, fx, fy);
    const double Vo = pair_V(t.x, r2, c.S[0], c.S[1], c.S[2], bx, by, bz, fx, fy);
    const double xn = beta * (Vn - t.y), xo = beta * (Vo - t.y);
    if (!(xn < 0.0) || !(xo < 0.0)) return 2;
    double Ln, Lo, sn, so;
    if (xn > -P.ln2_hi) {
      const double z = -expm1(xn);
      Ln = log(z);
      sn = (1.0 - z) / z;
    } else {
      const double y = exp(xn);
      Ln = log1p(-y);
      sn = 2.0 * y;
    }
    if (xo > -P.ln2_hi) {
      const double z = -expm1(xo);
      Lo = log(z);
      so = (1.0 - z) / z;
    } else {
      const double y = exp(xo);
      Lo = log1p(-y);
      so = 2.0 * y;
    }
    const double dbv = beta * (Vn - Vo);
    const double term = (dbv - Ln) + Lo;
    sum += term;
    sumabs += fabs(term);
    ++nterm;
    const double dV = 0x1p-47 * t.x * r2;
    const double dx0 = beta * (dV + 0x1p-52 * t.y);
    const double dxn = dx0 + 0x1p-52 * fabs(xn), dxo = dx0 + 0x1p-52 * fabs(xo);
    if (dxn > 0.25 * fabs(xn) || dxo > 0.25 * fabs(xo)) return 2;
    bnd += 2.0 * beta * dV + 0x1p-51 * fabs(dbv) + sn * dxn + so * dxo +
           0x1p-49 * (2.0 + fabs(Ln) + fabs(Lo)) + 0x1p-51 * (fabs(dbv) + fabs(Ln) + fabs(Lo));
  }
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
    const double tex = -(beta * P.J) * dot;
    sum += tex;
    sumabs += fabs(tex);
    ++nterm;
    bnd += 0x1p-44 * fabs(beta * P.J);
  }
  const double lu = log(c.u);
  const double mu = lu + sum;
  const double B = 2.0 * (bnd + (double)(nterm + 1) * 0x1p-52 * sumabs + 0x1p-50 * fabs(lu) +
                          0x1p-52 * fabs(mu));
  if (mu < -B) return 1;
  if (mu > B) return 0;
  return 2;
}

// FP32 screen: shadow spins (|dS| <= 2^-24 per component), FP32 table constants, CUDA's
// single-precision functions (<= 2 ulp; 4x margin) and a compensated (Neumaier) sum.
__device__ __forceinline__ int accept_fp32(const DevParams& P, const SiteCtx& c,
                                           const float4* __restrict__ xy32,
                                           const float* __restrict__ s32,
                                           const uint32_t* __restrict__ row_ptr,
                                           const uint32_t* __restrict__ col) {
  if (c.u < 0x1p-100) return 2;
  const float beta = (float)P.beta;
  const float ax = (float)c.S[0], ay = (float)c.S[1], az = (float)c.S[2];
  const float nx = (float)c.Sn[0], ny = (float)c.Sn[1], nz = (float)c.Sn[2];
  float sum = 0.f, comp = 0.f, sumabs = 0.f, bnd = 0.f;
  const float ln2 = 0.693147182f;  // fl32(ln 2): only the branch point of log1mexp
  for (uint32_t e = row_ptr[c.i]; e < row_ptr[c.i + 1]; ++e) {
    const uint32_t cj = col[e];
    if (cj & kExchOnly) continue;
    const int64_t j = cj;
    const int32_t dx = (int32_t)(j % P.Lx) - c.xi, dy = (int32_t)(j / P.Lx) - c.yi;
    const float4 t = __ldg(&xy32[(int64_t)(dx < 0 ? -dx : dx) + (int64_t)P.Lx * (dy < 0 ? -dy : dy)]);
    const float r2 = (float)(dx * dx + dy * dy);
    const float fx = (float)dx, fy = (float)dy;
    const float bx = s32[j], by = s32[P.N + j], bz = s32[2 * P.N + j];
    // per-edge field of the pair: f = Dc [r^2 S_j - 3 (S_j.d) d];  V(S) = S.f
    const float pb = bx * fx + by * fy;
    const float gx = t.x * (r2 * bx - 3.0f * pb * fx);
    const float gy = t.x * (r2 * by - 3.0f * pb * fy);
    const float gz = t.x * (r2 * bz);
    const float Vn = nx * gx + ny * gy + nz * gz;
    const float Vo = ax * gx + ay * gy + az * gz;
    const float xn = beta * (Vn - t.y), xo = beta * (Vo - t.y);
    if (!(xn < 0.f) || !(xo < 0.f)) return 2;
    float Ln, Lo, sn, so;
    if (xn > -ln2) {
      const float z = -expm1f(xn);
      Ln = logf(z);
      sn = (1.0f - z) / z;
    } else {
      const float y = expf(xn);
      Ln = log1pf(-y);
      sn = 2.0f * y;
    }
    if (xo > -ln2) {
      const float z = -expm1f(xo);
      Lo = logf(z);
      so = (1.0f - z) / z;
    } else {
      const float y = expf(xo);
      Lo = log1pf(-y);
      so = 2.0f * y;
    }
    const float dbv = beta * (Vn - Vo);
    const float term = (dbv - Ln) + Lo;
    // Neumaier compensated summation
    const float tsum = sum + term;
    comp += fabsf(sum) >= fabsf(term) ? (sum - tsum) + term : (term - tsum) + sum;
    sum = tsum;
    sumabs += fabsf(term);
    const float dV = 0x1p-16f * t.x * r2;  // |V error| incl. shadow spins and the field
    const float dx0 = beta * (dV + 0x1p-22f * t.y);
    const float dxn = dx0 + 0x1p-21f * fabsf(xn), dxo = dx0 + 0x1p-21f * fabsf(xo);
    if (dxn > 0.25f * fabsf(xn) || dxo > 0.25f * fabsf(xo)) return 2;
    bnd += 2.0f * beta * dV + 0x1p-21f * fabsf(dbv) + sn * dxn + so * dxo +
           0x1p-19f * (2.0f + fabsf(Ln) + fabsf(Lo)) + 0x1p-22f * (fabsf(dbv) + fabsf(Ln) + fabsf(Lo));
  }
  float tex = 0.f;
  if (P.J != 0.0) {
    float h0 = 0.f, h1 = 0.f, h2 = 0.f;
    const int64_t nb[4] = {c.xi > 0 ? c.i - 1 : -1, c.xi + 1 < P.Lx ? c.i + 1 : -1,
                           c.yi > 0 ? c.i - P.Lx : -1, c.yi + 1 < P.Ly ? c.i + P.Lx : -1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (nb[q] < 0) continue;
      h0 += s32[nb[q]];
      h1 += s32[P.N + nb[q]];
      h2 += s32[2 * P.N + nb[q]];
    }
    const float bj = (float)(P.beta * P.J);
    tex = -bj * ((nx - ax) * h0 + (ny - ay) * h1 + (nz - az) * h2);
    bnd += 0x1p-14f * fabsf(bj);
    sumabs += fabsf(tex);
  }
  const float lu = logf((float)c.u);
  const float mu = lu + ((sum + comp) + tex);
  const float B = 2.0f * (bnd + 0x1p-21f * sumabs + 0x1p-20f * fabsf(lu) + 0x1p-23f +
                          0x1p-23f * fabsf(mu));
  if (mu < -B) return 1;
  if (mu > B) return 0;
  return 2;
}

template <int PREC>
__global__ void __launch_bounds__(256) k_sweep(const DevParams P, const double2* __restrict__ xy,
                                               const float4* __restrict__ xy32,
                                               double* __restrict__ s, float* __restrict__ s32,
                                               const uint32_t* __restrict__ row_ptr,
                                               const uint32_t* __restrict__ col,
                                               const uint32_t* __restrict__ perm,
                                               const uint32_t* __restrict__ off, uint32_t colour,
                                               uint64_t step, uint8_t* __restrict__ acc,
                                               DevCounters* __restrict__ cnt) {
  const uint32_t b = off[colour], e = off[colour + 1];
  unsigned long long g64 = 0, g32 = 0;
  for (uint32_t idx = b + blockIdx.x * blockDim.x + threadIdx.x; idx < e;
       idx += gridDim.x * blockDim.x) {
    SiteCtx c;
    c.i = perm[idx];
    c.xi = (int32_t)(c.i % P.Lx);
    c.yi = (int32_t)(c.i / P.Lx);
    c.S[0] = s[c.i];
    c.S[1] = s[P.N + c.i];
    c.S[2] = s[2 * P.N + c.i];
    bool found = false;
    for (uint64_t a = 0; a < 64 && !found; ++a) {
      const W4 w = philox((uint64_t)c.i, step, a, kTagPropose, P.key0, P.key1);
      if (marsaglia(w.w[0], w.w[1], c.Sn[0], c.Sn[1], c.Sn[2])) {
        c.u = u53(w.w[2]);
        found = true;
      }
    }
    bool ok = false;
    if (found) {
      if (c.u == 0.0) {
        ok = true;
      } else {
        int d = 2;
        if (PREC == 1) {
          d = accept_fp32(P, c, xy32, s32, row_ptr, col);
          if (d == 2) ++g32;
        }
        if (d == 2) d = accept_fp64(P, c, xy, s, row_ptr, col);
        if (d == 2) {
          ++g64;
          d = accept_dd(P, c, s, row_ptr, col) ? 1 : 0;
        }
        ok = d == 1;
      }
    }
    if (ok) {
      s[c.i] = c.Sn[0];
      s[P.N + c.i] = c.Sn[1];
      s[2 * P.N + c.i] = c.Sn[2];
      if (PREC == 1) {
        s32[c.i] = (float)c.Sn[0];
        s32[P.N + c.i] = (float)c.Sn[1];
        s32[2 * P.N + c.i] = (float)c.Sn[2];
      }
    }
    acc[c.i] = ok ? 1 : 0;
  }
  g64 = warp_sum_u64(g64);
  g32 = warp_sum_u64(g32);
  if ((threadIdx.x & 31) == 0) {
    if (g64) atomicAdd(&cnt->guard_fp64, g64);
    if (g32) atomicAdd(&cnt->guard_fp32, g32);
  }
}

}  // namespace

cudaError_t sweep_run(const DevParams& P, const Table& t, double* s, float* s32,
                      const uint32_t* row_ptr, const uint32_t* col, const uint32_t* perm,
                      const uint32_t* off, uint32_t g, uint64_t step, int precision,
                      uint8_t* acc, DevCounters* cnt, cudaStream_t st, int64_t* launches) {
  // one launch per colour in ascending order; a class holds about N / g sites
  const int64_t per = P.N / (g > 0 ? g : 1) + 1;
  int64_t nb = (per + 255) / 256;
  const int64_t cap = 8 * (int64_t)num_sms();
  if (nb > cap) nb = cap;
  if (nb < 1) nb = 1;
  for (uint32_t c = 0; c < g; ++c) {
    if (precision == 1)
      k_sweep<1><<<(unsigned)nb, 256, 0, st>>>(P, t.xy, t.xy32, s, s32, row_ptr, col, perm, off,
                                                c, step, acc, cnt);
    else
      k_sweep<0><<<(unsigned)nb, 256, 0, st>>>(P, t.xy, t.xy32, s, s32, row_ptr, col, perm, off,
                                                c, step, acc, cnt);
    ++*launches;
  }
  return cudaGetLastError();
}

}  // namespace sco
