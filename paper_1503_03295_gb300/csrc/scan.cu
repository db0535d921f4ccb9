// scan.cu -- device prefix sums used to turn counts into offsets: per-site degrees into
// CSR row pointers, r^2 bucket counts into bucket starts, hazards into the prefix W.
// Three passes over tiles of kTile elements: tile totals, a scan of the totals, and a
// scan of every tile from its offset.  Totals are accumulated in 64 bits.
#include <cstdint>

#include "sco_internal.h"

namespace sco {

namespace {

constexpr int kThreads = 512;
constexpr int kPer = 8;
constexpr int kTile = kThreads * kPer;

template <typename T>
__device__ __forceinline__ T warp_incl(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Inclusive scan of one value per thread across the block; returns the block total too.
template <typename T>
__device__ __forceinline__ T block_incl(T v, T* warp_tot, T& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_incl(v);
  if (lane == 31) warp_tot[wid] = v;
  __syncthreads();
  if (wid == 0) {
    T w = lane < (kThreads / 32) ? warp_tot[lane] : T(0);
    w = warp_incl(w);
    if (lane < (kThreads / 32)) warp_tot[lane] = w;
  }
  __syncthreads();
  if (wid > 0) v += warp_tot[wid - 1];
  total = warp_tot[kThreads / 32 - 1];
  __syncthreads();
  return v;
}

template <typename Tin>
__global__ void __launch_bounds__(kThreads) k_tile_sums(const Tin* __restrict__ in, int64_t n,
                                                         uint64_t* __restrict__ sums) {
  __shared__ uint64_t wt[kThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kTile;
  uint64_t acc = 0;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int64_t idx = base + (int64_t)k * kThreads + threadIdx.x;
    if (idx < n) acc += (uint64_t)in[idx];
  }
  uint64_t total;
  block_incl<uint64_t>(acc, wt, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Exclusive scan of the tile totals (one block, serial over chunks); total at sums[nt].
__global__ void __launch_bounds__(kThreads) k_scan_sums(uint64_t* __restrict__ sums, int64_t nt) {
  __shared__ uint64_t wt[kThreads / 32];
  uint64_t carry = 0;
  for (int64_t b = 0; b < nt; b += kThreads) {
    const int64_t idx = b + threadIdx.x;
    const uint64_t v = idx < nt ? sums[idx] : 0;
    uint64_t total;
    const uint64_t inc = block_incl<uint64_t>(v, wt, total);
    if (idx < nt) sums[idx] = carry + inc - v;
    carry += total;
  }
  if (threadIdx.x == 0) sums[nt] = carry;
}

template <typename Tin, typename Tout, bool kInclusive>
__global__ void __launch_bounds__(kThreads) k_tile_scan(const Tin* __restrict__ in, int64_t n,
                                                         const uint64_t* __restrict__ sums,
                                                         Tout* __restrict__ out) {
  __shared__ uint64_t wt[kThreads / 32];
  __shared__ uint64_t carry_s;
  const int64_t base = (int64_t)blockIdx.x * kTile;
  if (threadIdx.x == 0) carry_s = sums[blockIdx.x];
  __syncthreads();
  uint64_t carry = carry_s;
  for (int k = 0; k < kPer; ++k) {
    const int64_t idx = base + (int64_t)k * kThreads + threadIdx.x;
    const uint64_t v = idx < n ? (uint64_t)in[idx] : 0;
    uint64_t total;
    const uint64_t inc = block_incl<uint64_t>(v, wt, total);
    if (idx < n) out[idx] = (Tout)(carry + (kInclusive ? inc : inc - v));
    carry += total;
  }
}

}  // namespace

size_t scan_tmp_bytes(int64_t n) { return (size_t)((n + kTile - 1) / kTile + 2) * 8; }

template <typename Tin, typename Tout, bool kInclusive>
static cudaError_t scan_impl(const Tin* in, Tout* out, int64_t n, uint64_t* tmp,
                             uint64_t* total_dev, cudaStream_t s, int64_t* launches) {
  const int64_t nt = (n + kTile - 1) / kTile;
  if (nt > 0) {
    k_tile_sums<Tin><<<(unsigned)nt, kThreads, 0, s>>>(in, n, tmp);
    ++*launches;
  }
  k_scan_sums<<<1, kThreads, 0, s>>>(tmp, nt);
  ++*launches;
  if (nt > 0) {
    k_tile_scan<Tin, Tout, kInclusive><<<(unsigned)nt, kThreads, 0, s>>>(in, n, tmp, out);
    ++*launches;
  }
  if (total_dev) {
    cudaError_t e = cudaMemcpyAsync(total_dev, tmp + nt, 8, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t scan_excl_u32(const uint32_t* in, uint32_t* out, int64_t n, uint64_t* tmp,
                          uint64_t* total_dev, cudaStream_t s, int64_t* launches) {
  return scan_impl<uint32_t, uint32_t, false>(in, out, n, tmp, total_dev, s, launches);
}

cudaError_t scan_incl_u64(const uint64_t* in, uint64_t* out, int64_t n, uint64_t* tmp,
                          uint64_t* total_dev, cudaStream_t s, int64_t* launches) {
  return scan_impl<uint64_t, uint64_t, true>(in, out, n, tmp, total_dev, s, launches);
}

}  // namespace sco
