// sweep.cu -- step (B) of Sec. 2.1 / step (3) of Fig. 1 for one lattice: Metropolis
// updates of all sites of one colour class at a time (one launch per colour), with the
// undecided sites settled afterwards by one warp each.  Sites of one colour share no pair,
// so they update independently.  The per-site decision is in sweep_dev.cuh.
#include <cstdint>

#include "sweep_dev.cuh"
#include "switch_dev.cuh"

namespace sco {

namespace {

// Draws the proposal of every site for MC step `step` (see take_proposal); with the pair cache,
// marks every site as not decided yet in this step, keeping its acceptance parity unless the
// cache was just written from the spins (reset).
__global__ void __launch_bounds__(256) k_propose(const DevParams P, uint64_t step,
                                                 double4_32a* __restrict__ prop,
                                                 uint8_t* __restrict__ upd, int reset) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= P.N) return;
  if (upd) upd[i] = reset ? 0 : upd[i] & 4u;
  SiteCtx c;
  c.i = i;
  const bool ok = propose(P, c, step);
  prop[i] = ok ? make_double4_32a(c.Sn[0], c.Sn[1], c.Sn[2], c.u)
               : make_double4_32a(0.0, 0.0, 1.0, -1.0);
}

// In the FP64 form, classes of at most this many sites (the largest colours hold a few dozen)
// are left to k_resolve, which sweeps them one warp per site: the pairs of a site spread over
// the lanes, the launch lasts about one pair's FP64 chain instead of a whole row's.
constexpr uint32_t kSweepWarpSites = 4096;

// One thread per site of the class.  A site whose decision stays inside the error bound is
// appended to the deferred list of the colour and settled by k_resolve (one warp per site),
// so that no thread of this kernel runs the long FP64 / double-double evaluations.
// CACHE (FP64 form only): old-spin pair terms from the pair cache (see PairCache).
template <int PREC, bool CACHE>
__global__ void __launch_bounds__(128, 8) k_sweep(const DevParams P, const Sw64* __restrict__ sw,
                                               const float4* __restrict__ sw32,
                                               double* __restrict__ s, float4* __restrict__ s32,
                                               const uint32_t* __restrict__ row_ptr,
                                               const uint32_t* __restrict__ col,
                                               const uint32_t* __restrict__ perm,
                                               const uint32_t* __restrict__ off, uint32_t colour,
                                               const double4_32a* __restrict__ prop,
                                               uint8_t* __restrict__ acc,
                                               uint32_t* __restrict__ defer,
                                               uint32_t* __restrict__ dcnt,
                                               DevCounters* __restrict__ cnt, PairCache pc) {
  const uint32_t b = off[colour], e = off[colour + 1];
  if (PREC == 0 && e - b <= kSweepWarpSites) return;  // swept by k_resolve
  unsigned long long nd = 0;
  for (uint32_t idx = b + blockIdx.x * blockDim.x + threadIdx.x; idx < e;
       idx += gridDim.x * blockDim.x) {
    SiteCtx c;
    load_site(P, c, perm[idx], s);
    const uint32_t ui = CACHE ? pc.upd[c.i] : 0u;
    if (!take_proposal(c, prop)) {
      acc[c.i] = 0;
      if (CACHE) pc.upd[c.i] = upd_decided(ui, false);
      continue;
    }
    int d = 1;
    if (CACHE) {
      // evaluated also when u = 0 (accepted outright): the proposed-spin terms must be written
      d = accept_fp64_cached(P, c, sw, s, row_ptr, col, pc, ui);
      if (c.u == 0.0) d = 1;
    } else if (c.u != 0.0) {
      d = PREC == 1 ? accept_fp32(P, c, sw32, s32, row_ptr, col)
                    : accept_fp64(P, c, sw, s, row_ptr, col);
    }
    if (d == 2) {
      defer[b + atomicAdd(&dcnt[colour], 1u)] = (uint32_t)c.i;
      ++nd;
      continue;
    }
    write_site(P, c, d == 1, s, PREC == 1 ? s32 : nullptr, acc);
    if (CACHE) pc.upd[c.i] = upd_decided(ui, d == 1);
  }
  nd = warp_sum_u64(nd);
  if ((threadIdx.x & 31) == 0 && nd) {
    if (PREC == 1) atomicAdd(&cnt->guard_fp32, nd);
    else atomicAdd(&cnt->guard_fp64, nd);
  }
}

// Settles the deferred sites of a colour: one warp per site, FP64 then double-double.  In the
// FP64 form a class of at most kSweepWarpSites sites is swept here whole, one warp per site.
__global__ void __launch_bounds__(128) k_resolve(const DevParams P, const Sw64* __restrict__ sw,
                                                 double* __restrict__ s, float4* __restrict__ s32,
                                                 const uint32_t* __restrict__ row_ptr,
                                                 const uint32_t* __restrict__ col,
                                                 const uint32_t* __restrict__ perm,
                                                 const uint32_t* __restrict__ off,
                                                 const uint32_t* __restrict__ defer,
                                                 const uint32_t* __restrict__ dcnt, uint32_t colour,
                                                 const double4_32a* __restrict__ prop,
                                                 int fp32_screened,
                                                 uint8_t* __restrict__ acc,
                                                 DevCounters* __restrict__ cnt, PairCache pc) {
  const bool cache = pc.hid != nullptr;  // FP64 form with the pair cache (uniform)
  const uint32_t b = off[colour], e = off[colour + 1];
  const bool whole = !fp32_screened && e - b <= kSweepWarpSites;  // uniform
  const uint32_t n = whole ? e - b : dcnt[colour];
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned long long ndd = 0;
  for (uint32_t q = warp; q < n; q += nwarps) {
    SiteCtx c;
    load_site(P, c, whole ? perm[b + q] : defer[b + q], s);
    const uint32_t ui = cache ? pc.upd[c.i] : 0u;
    if (!take_proposal(c, prop)) {  // only a whole-class site can lack a move
      if (lane == 0) {
        acc[c.i] = 0;
        if (cache) pc.upd[c.i] = upd_decided(ui, false);
      }
      __syncwarp();
      continue;
    }
    int d = 2;
    if (cache && whole) {
      // the proposed-spin terms are written even when u = 0 accepts outright (deferred sites
      // had them written by k_sweep)
      d = accept_fp64_warp_cached(P, c, sw, s, row_ptr, col, pc, ui, lane);
      if (c.u == 0.0) d = 1;
    } else if (whole && c.u == 0.0) {
      d = 1;
    } else if (fp32_screened || whole) {
      d = accept_fp64_warp(P, c, sw, s, row_ptr, col, lane);
    }
    if (d == 2) {
      ++ndd;
      d = accept_dd_warp(P, c, s, row_ptr, col, lane) ? 1 : 0;
    }
    if (lane == 0) {
      write_site(P, c, d == 1, s, fp32_screened ? s32 : nullptr, acc);
      if (cache) pc.upd[c.i] = upd_decided(ui, d == 1);
    }
    __syncwarp();
  }
  // deferred FP64-form sites were counted by k_sweep already
  if (lane == 0 && ndd && (fp32_screened || whole)) atomicAdd(&cnt->guard_fp64, ndd);
}

// Pair cache from scratch at the current spins (after the spins changed outside the sweep): the
// FP64 term of every surviving dipolar pair, evaluated as the switch does.
__device__ __forceinline__ void cache_build(const DevParams& P, const Sw64* __restrict__ sw,
                                            const double* __restrict__ s, uint32_t i, uint32_t jv,
                                            uint32_t h, double4_32a* keep) {
  if (jv & kExchOnly) return;
  const uint32_t j = jv & kIndexMask;
  const uint32_t yi = site_row(i, P), yj = site_row(j, P);
  const int32_t dx = (int32_t)(j - yj * (uint32_t)P.Lx) - (int32_t)(i - yi * (uint32_t)P.Lx);
  const int32_t dy = (int32_t)yj - (int32_t)yi;
  const double Si[3] = {s[i], s[P.N + i], s[2 * P.N + i]};
  const double Sj[3] = {s[j], s[P.N + j], s[2 * P.N + j]};
  double x;
  const double z = pair_keep64(
      sw[(int64_t)(dx < 0 ? -dx : dx) + (int64_t)P.Lx * (dy < 0 ? -dy : dy)], Si, Sj, dx, dy, &x);
  reinterpret_cast<double2*>(&keep[h])[0] = make_double2(z, x);
}

__global__ void __launch_bounds__(256) k_cache_build(const DevParams P, const Sw64* __restrict__ sw,
                                                     const double* __restrict__ s,
                                                     const uint32_t* __restrict__ hslot,
                                                     const uint32_t* __restrict__ hcnt,
                                                     const uint32_t* __restrict__ ovf,
                                                     const DevCounters* __restrict__ cnt,
                                                     uint32_t ovf_cap, double4_32a* keep) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < P.N) {
    const uint32_t n = min(hcnt[i], (uint32_t)kSlotCap);
    for (uint32_t q = 0; q < n; ++q) {
      const uint32_t h = (uint32_t)i * (uint32_t)kSlotCap + q;
      cache_build(P, sw, s, (uint32_t)i, hslot[h], h, keep);
    }
  }
  const unsigned long long no = min(cnt->ovf_n, (unsigned long long)ovf_cap);
  for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < no;
       q += (unsigned long long)gridDim.x * blockDim.x)
    cache_build(P, sw, s, ovf[2 * q], ovf[2 * q + 1], (uint32_t)P.N * (uint32_t)kSlotCap + (uint32_t)q,
                keep);
}

}  // namespace

cudaError_t cache_build_run(const DevParams& P, const Table& t, const double* s,
                            const SwitchBufs& b, const DevCounters* cnt, cudaStream_t st,
                            int64_t* launches) {
  k_cache_build<<<(unsigned)((P.N + 255) / 256), 256, 0, st>>>(P, t.sw64, s, b.hslot, b.hcnt, b.ovf,
                                                               cnt, b.ovf_cap, b.keep);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t sweep_run(const DevParams& P, const Table& t, double* s, float4* s32,
                      const uint32_t* row_ptr, const uint32_t* col, const uint32_t* perm,
                      const uint32_t* off, uint32_t g, uint64_t step, int precision,
                      uint8_t* acc, uint32_t* defer, uint32_t* dcnt, double4_32a* prop,
                      DevCounters* cnt, const PairCache& pc, cudaStream_t st,
                      int64_t* launches) {
  cudaError_t e = cudaMemsetAsync(dcnt, 0, (size_t)g * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  const bool cache = precision == 0 && pc.hid != nullptr;
  k_propose<<<(unsigned)((P.N + 255) / 256), 256, 0, st>>>(P, step, prop, cache ? pc.upd : nullptr,
                                                           pc.reset);
  ++*launches;
  const unsigned nres = (unsigned)(4 * num_sms());
  // one launch per colour in ascending order; a class holds about N / g sites.  The grid is a
  // whole number of blocks per SM (every SM gets the same share of a class: the FP64 form is
  // bound by each SM's FP64 pipe) and at most the resident 8 per SM of __launch_bounds__.
  const int64_t per = P.N / (g > 0 ? g : 1) + 1;
  const int64_t sms = num_sms();
  int64_t nb = (per + 127) / 128;
  nb = (nb + sms - 1) / sms * sms;
  // the FP32-guarded form measured faster with every resident block (2.48 -> 2.42 ms per step
  // at L = 2304), the FP64 form slower (7.09 -> 7.53 ms)
  if (nb > 8 * sms || precision == 1) nb = 8 * sms;
  if (nb < 1) nb = 1;
  for (uint32_t c = 0; c < g; ++c) {
    if (precision == 1)
      k_sweep<1, false><<<(unsigned)nb, 128, 0, st>>>(P, t.sw64, t.sw32, s, s32, row_ptr, col,
                                                       perm, off, c, prop, acc, defer, dcnt, cnt,
                                                       pc);
    else if (cache)
      k_sweep<0, true><<<(unsigned)nb, 128, 0, st>>>(P, t.sw64, t.sw32, s, s32, row_ptr, col, perm,
                                                      off, c, prop, acc, defer, dcnt, cnt, pc);
    else
      k_sweep<0, false><<<(unsigned)nb, 128, 0, st>>>(P, t.sw64, t.sw32, s, s32, row_ptr, col,
                                                       perm, off, c, prop, acc, defer, dcnt, cnt,
                                                       pc);
    k_resolve<<<nres, 128, 0, st>>>(P, t.sw64, s, s32, row_ptr, col, perm, off, defer, dcnt, c,
                                    prop, precision == 1 ? 1 : 0, acc, cnt,
                                    cache ? pc : PairCache{});
    *launches += 2;
  }
  return cudaGetLastError();
}

}  // namespace sco
