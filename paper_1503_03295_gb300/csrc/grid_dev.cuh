// grid_dev.cuh -- small device helpers shared by the persistent (cooperative) kernels: a
// bounded grid-wide barrier, L2-coherent loads, a block-wide scan and a sorted-array search.
#pragma once

#include <cstdint>

#include "kw_dev.cuh"

namespace sco {
namespace {

// Largest r in [0, n) with a[r] <= x (a[0] <= x, a non-decreasing).
__device__ __forceinline__ int find_le(const uint32_t* a, int n, uint32_t x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int m = (lo + hi + 1) >> 1;
    if (a[m] <= x) lo = m;
    else hi = m - 1;
  }
  return lo;
}

__device__ __forceinline__ uint32_t ld_u32_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier of a cooperative launch (all blocks resident).  bar[0] is an arrival
// counter: block 0 adds 2^31 - (blocks - 1) and every other block 1, so the top bit flips
// exactly when the last block arrives and the low bits return to where they were; a block
// waits for the flip of the bit it saw when it arrived.  The wait is bounded: after ns_limit,
// or once another block reported an error, the block gives up, sets SCO_ETIMEOUT in *status
// and returns false.  Also false when *status holds an error after the barrier.
__device__ __noinline__ bool grid_sync(unsigned* bar, int* status, unsigned long long ns_limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1) : 1u;
    __threadfence();
    const unsigned old = atomicAdd(&bar[0], inc);
    if (((old + inc) ^ old) & 0x80000000u) {
      // last to arrive: nothing to wait for
    } else {
      const unsigned long long t0 = global_ns();
      unsigned spins = 0;
      while (((ld_acquire_u32(&bar[0]) ^ old) & 0x80000000u) == 0) {
        __nanosleep(20);
        if ((++spins & wait_spin_mask(ns_limit)) == 0 && (global_ns() - t0 > ns_limit || ld_status(status) != 0)) {
          atomicCAS(status, 0, kStatusTimeout);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok && ld_status(status) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// The same barrier in two halves, so that a block can do independent work (prefetches)
// between its arrival and its wait.  Every thread calls both; the block's earlier writes are
// published by the arrival.
__device__ __forceinline__ void grid_arrive(unsigned* bar, unsigned* s_old) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1) : 1u;
    __threadfence();
    const unsigned old = atomicAdd(&bar[0], inc);
    // remember the top bit to wait for a change of; 0xFFFFFFFF: this block arrived last
    s_old[0] = (((old + inc) ^ old) & 0x80000000u) ? 0xFFFFFFFFu : (old & 0x80000000u);
  }
}
__device__ __noinline__ bool grid_wait(unsigned* bar, const unsigned* s_old, int* status,
                                       unsigned long long ns_limit) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned old = s_old[0];
    if (old != 0xFFFFFFFFu) {
      const unsigned long long t0 = global_ns();
      unsigned spins = 0;
      while (((ld_acquire_u32(&bar[0]) ^ old) & 0x80000000u) == 0) {
        __nanosleep(20);
        if ((++spins & wait_spin_mask(ns_limit)) == 0 && (global_ns() - t0 > ns_limit || ld_status(status) != 0)) {
          atomicCAS(status, 0, kStatusTimeout);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok && ld_status(status) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ void smem_copy(void* dst, const void* src, int bytes) {
  for (int k = threadIdx.x; k < bytes / 4; k += blockDim.x)
    static_cast<uint32_t*>(dst)[k] = static_cast<const uint32_t*>(src)[k];
}

// Exclusive scan of a[0..n) in place, a[n] = total; blockDim.x == 256, n <= 256 * 8.
__device__ void block_scan_excl(uint32_t* a, int n) {
  __shared__ uint32_t wsum[8];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int per = (n + 255) / 256;  // <= 8 consecutive entries per thread
  uint32_t v[8], s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int q = per * t + k;
    v[k] = (k < per && q < n) ? a[q] : 0u;
    s += v[k];
  }
  uint32_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  uint32_t run = x - s;
  for (int k = 0; k < w; ++k) run += wsum[k];
  uint32_t total = 0;
  for (int k = 0; k < 8; ++k) total += wsum[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int q = per * t + k;
    if (k < per && q < n) a[q] = run;
    run += v[k];
  }
  if (t == 0) a[n] = total;
  __syncthreads();
}

}  // namespace
}  // namespace sco
