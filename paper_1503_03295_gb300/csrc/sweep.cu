// sweep.cu -- step (B) of Sec. 2.1 / step (3) of Fig. 1 for one lattice: Metropolis
// updates of all sites of one colour class at a time (one launch per colour), with the
// undecided sites settled afterwards by one warp each.  Sites of one colour share no pair,
// so they update independently.  The per-site decision is in sweep_dev.cuh.
#include <cstdint>

#include "sweep_dev.cuh"

namespace sco {

namespace {

// Draws the proposal of every site for MC step `step` (see take_proposal).
__global__ void __launch_bounds__(256) k_propose(const DevParams P, uint64_t step,
                                                 double4_32a* __restrict__ prop) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= P.N) return;
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
template <int PREC>
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
                                               DevCounters* __restrict__ cnt) {
  const uint32_t b = off[colour], e = off[colour + 1];
  if (PREC == 0 && e - b <= kSweepWarpSites) return;  // swept by k_resolve
  unsigned long long nd = 0;
  for (uint32_t idx = b + blockIdx.x * blockDim.x + threadIdx.x; idx < e;
       idx += gridDim.x * blockDim.x) {
    SiteCtx c;
    load_site(P, c, perm[idx], s);
    if (!take_proposal(c, prop)) {
      acc[c.i] = 0;
      continue;
    }
    int d = 1;
    if (c.u != 0.0) {
      d = PREC == 1 ? accept_fp32(P, c, sw32, s32, row_ptr, col)
                    : accept_fp64(P, c, sw, s, row_ptr, col);
    }
    if (d == 2) {
      defer[b + atomicAdd(&dcnt[colour], 1u)] = (uint32_t)c.i;
      ++nd;
      continue;
    }
    write_site(P, c, d == 1, s, PREC == 1 ? s32 : nullptr, acc);
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
                                                 DevCounters* __restrict__ cnt) {
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
    if (!take_proposal(c, prop)) {  // only a whole-class site can lack a move
      if (lane == 0) acc[c.i] = 0;
      __syncwarp();
      continue;
    }
    int d = 2;
    if (whole && c.u == 0.0) d = 1;
    else if (fp32_screened || whole) d = accept_fp64_warp(P, c, sw, s, row_ptr, col, lane);
    if (d == 2) {
      ++ndd;
      d = accept_dd_warp(P, c, s, row_ptr, col, lane) ? 1 : 0;
    }
    if (lane == 0) write_site(P, c, d == 1, s, fp32_screened ? s32 : nullptr, acc);
    __syncwarp();
  }
  // deferred FP64-form sites were counted by k_sweep already
  if (lane == 0 && ndd && (fp32_screened || whole)) atomicAdd(&cnt->guard_fp64, ndd);
}

}  // namespace

cudaError_t sweep_run(const DevParams& P, const Table& t, double* s, float4* s32,
                      const uint32_t* row_ptr, const uint32_t* col, const uint32_t* perm,
                      const uint32_t* off, uint32_t g, uint64_t step, int precision,
                      uint8_t* acc, uint32_t* defer, uint32_t* dcnt, double4_32a* prop,
                      DevCounters* cnt, cudaStream_t st, int64_t* launches) {
  cudaError_t e = cudaMemsetAsync(dcnt, 0, (size_t)g * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  k_propose<<<(unsigned)((P.N + 255) / 256), 256, 0, st>>>(P, step, prop);
  ++*launches;
  const unsigned nres = (unsigned)(4 * num_sms());
  // one launch per colour in ascending order; a class holds about N / g sites.  The grid is a
  // whole number of blocks per SM (every SM gets the same share of a class: the FP64 form is
  // bound by each SM's FP64 pipe) and at most the resident 8 per SM of __launch_bounds__.
  const int64_t per = P.N / (g > 0 ? g : 1) + 1;
  const int64_t sms = num_sms();
  int64_t nb = (per + 127) / 128;
  nb = (nb + sms - 1) / sms * sms;
  if (nb > 8 * sms) nb = 8 * sms;
  if (nb < 1) nb = 1;
  for (uint32_t c = 0; c < g; ++c) {
    if (precision == 1)
      k_sweep<1><<<(unsigned)nb, 128, 0, st>>>(P, t.sw64, t.sw32, s, s32, row_ptr, col, perm,
                                                off, c, prop, acc, defer, dcnt, cnt);
    else
      k_sweep<0><<<(unsigned)nb, 128, 0, st>>>(P, t.sw64, t.sw32, s, s32, row_ptr, col, perm,
                                                off, c, prop, acc, defer, dcnt, cnt);
    k_resolve<<<nres, 128, 0, st>>>(P, t.sw64, s, s32, row_ptr, col, perm, off, defer, dcnt, c,
                                    prop, precision == 1 ? 1 : 0, acc, cnt);
    *launches += 2;
  }
  return cudaGetLastError();
}

}  // namespace sco
