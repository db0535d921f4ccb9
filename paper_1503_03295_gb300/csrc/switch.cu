// switch.cu -- step (A) of Sec. 2.1 (potential switching) for one lattice and the
// compaction of the surviving pairs into a symmetric CSR graph.  The per-site body (bound
// thinning over the sorted half-plane list, exact decisions) is in switch_dev.cuh.
#include <cstdint>

#include "switch_dev.cuh"

namespace sco {

namespace {

// Persistent: each warp claims 32 sites at a time from a global counter, and a lane whose walk
// ends takes up the next claimed site at once, so that the lanes of a warp stay busy although
// the number of candidates differs from site to site (Poisson, mean about 14 at T = 0.6D).
// Five blocks per SM for the FP32-screened form (48 registers); four for the FP64 form, which
// takes the same time there with half the register spills.
template <int PREC>
__global__ void __launch_bounds__(256, PREC == 1 ? 5 : 4) k_switch(const DevParams P, const uint64_t* __restrict__ W,
                                                const uint64_t* __restrict__ Eb,
                                                const uint32_t* __restrict__ disp,
                                                const Sw64* __restrict__ sw64,
                                                const double* __restrict__ xyq,
                                                const float4* __restrict__ xy32,
                                                const double* __restrict__ s,
                                                const float4* __restrict__ s32, uint32_t epoch,
                                                int32_t mnn0, int32_t mnn1, SwitchBufs b,
                                                DevCounters* __restrict__ cnt) {
  // the head of the list: W (FP32-screened search) or the decay bits (FP64 search)
  __shared__ uint64_t sX[kNear];
  __shared__ uint32_t sD[kNear];
  const bool decay = PREC == 0 && Eb != nullptr;
  const int64_t nnear = P.K < kNear ? P.K : kNear;
  for (int q = threadIdx.x; q < nnear; q += blockDim.x) {
    sX[q] = decay ? Eb[q] : W[q];
    sD[q] = disp[q];
  }
  __syncthreads();
  NearTable T{sX, sD, W, disp, nnear, P.K, nnear};
  if (decay) {
    T.nw = 0;
    T.sE = sX;
    T.E = Eb;
    T.elast = P.K > 0 ? __ldg(&Eb[P.K - 1]) : 0ull;
  }
  const uint64_t Wtot = P.K > 0 ? __ldg(&W[P.K - 1]) : 0;
  SwitchOut o{b.hslot, b.indeg, b.ovf, b.ovf_cap, &cnt->ovf_n, &cnt->ovf_full};
  if (PREC == 0 && b.keep) {
    o.keep = b.keep;
    o.keep_ovf = b.keep + (size_t)P.N * kSlotCap;
  }
  const uint32_t N = (uint32_t)P.N;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned below = (1u << lane) - 1u;
  unsigned long long n_half = 0, n_dip = 0;
  unsigned ghits = 0, g32 = 0;
  SiteWalk<PREC> a;
  bool active = false, drained = false;  // drained, pool and pool_n are warp-uniform
  uint32_t pool = 0, pool_n = 0;
  for (;;) {
    unsigned need = __ballot_sync(0xffffffffu, !active);
    while (need != 0u && !drained) {
      if (pool_n == 0u) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&cnt->sw_next, 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= N) {
          drained = true;
          break;
        }
        pool = base;
        pool_n = min(32u, N - base);
      }
      const uint32_t take = min((uint32_t)__popc(need), pool_n);
      const uint32_t rank = (uint32_t)__popc(need & below);
      if (!active && rank < take) {
        walk_begin<PREC>(P, T, s, s32, pool + rank, pool + rank, a);
        active = true;
      }
      pool += take;
      pool_n -= take;
      need = __ballot_sync(0xffffffffu, !active);
    }
    const unsigned act = __ballot_sync(0xffffffffu, active);
    if (act == 0u) break;
    if (active && !walk_step<PREC>(P, T, Wtot, sw64, xyq, xy32, s, s32, epoch, mnn0, mnn1, o,
                                   a, n_dip, ghits, g32, act)) {
      const uint32_t n_out = walk_end<PREC>(P, mnn0, mnn1, o, a);
      b.hcnt[a.i] = n_out;
      n_half += n_out;
      active = false;
    }
  }
  n_half = warp_sum_u64(n_half);
  n_dip = warp_sum_u64(n_dip);
  const unsigned long long gh = warp_sum_u64(ghits), gl = warp_sum_u64(g32);
  if ((threadIdx.x & 31) == 0) {
    if (n_half) atomicAdd(&cnt->n_half, n_half);
    if (n_dip) atomicAdd(&cnt->n_dip, n_dip);
    if (gh) atomicAdd(&cnt->guard_fp64, gh);
    if (gl) atomicAdd(&cnt->guard_fp32, gl);
  }
}

__global__ void k_degree(int64_t N, const uint32_t* __restrict__ hcnt,
                         const uint32_t* __restrict__ indeg, uint32_t* __restrict__ deg,
                         DevCounters* __restrict__ cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  unsigned m = 0;
  if (i < N) {
    m = hcnt[i] + indeg[i];
    deg[i] = m;
  } else if (i == N) {
    deg[N] = 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(&cnt->max_degree, m);
}

// Row i holds its lower neighbours (j < i, scattered here by the sites j) followed by its
// upper neighbours (written by site i from its slots).  Rows are sorted afterwards.
// hid (optional): both entries of a pair get the half-edge id i * kSlotCap + q.
__global__ void k_fill(int64_t N, const uint32_t* __restrict__ hslot,
                       const uint32_t* __restrict__ hcnt, const uint32_t* __restrict__ indeg,
                       const uint32_t* __restrict__ row_ptr, uint32_t* __restrict__ lcur,
                       uint32_t* __restrict__ col, uint32_t* __restrict__ hid) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const uint32_t n = min(hcnt[i], (uint32_t)kSlotCap);
  const uint32_t up = row_ptr[i] + indeg[i];
  // eight half-edges at a time: their slot and row-pointer loads, then their atomics, then their
  // stores, each group issued together (the atomics' returns were the chain)
  constexpr uint32_t kB = 8;
  for (uint32_t q0 = 0; q0 < n; q0 += kB) {
    uint32_t jv[kB], base[kB], lo[kB];
#pragma unroll
    for (uint32_t a = 0; a < kB; ++a)
      jv[a] = q0 + a < n ? hslot[i * (int64_t)kSlotCap + q0 + a] : 0u;
#pragma unroll
    for (uint32_t a = 0; a < kB; ++a) base[a] = q0 + a < n ? row_ptr[jv[a] & kIndexMask] : 0u;
#pragma unroll
    for (uint32_t a = 0; a < kB; ++a)
      lo[a] = q0 + a < n ? base[a] + atomicAdd(&lcur[jv[a] & kIndexMask], 1u) : 0u;
#pragma unroll
    for (uint32_t a = 0; a < kB; ++a) {
      if (q0 + a >= n) continue;
      col[up + q0 + a] = jv[a];
      col[lo[a]] = (uint32_t)i | (jv[a] & kExchOnly);
      if (hid) {
        const uint32_t h = (uint32_t)i * (uint32_t)kSlotCap + q0 + a;
        hid[up + q0 + a] = h;
        hid[lo[a]] = h;
      }
    }
  }
}

// Overflow half-edge q: id N * kSlotCap + q.
__global__ void k_fill_ovf(unsigned long long n, uint32_t N, const uint32_t* __restrict__ ovf,
                           const uint32_t* __restrict__ indeg,
                           const uint32_t* __restrict__ row_ptr, uint32_t* __restrict__ lcur,
                           uint32_t* __restrict__ ocur, uint32_t* __restrict__ col,
                           uint32_t* __restrict__ hid) {
  const unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  if (q >= n) return;
  const uint32_t i = ovf[2 * q], jv = ovf[2 * q + 1];
  const uint32_t j = jv & kIndexMask;
  const uint32_t up = row_ptr[i] + indeg[i] + kSlotCap + atomicAdd(&ocur[i], 1u);
  const uint32_t lo = row_ptr[j] + atomicAdd(&lcur[j], 1u);
  col[up] = jv;
  col[lo] = i | (jv & kExchOnly);
  if (hid) {
    const uint32_t h = N * (uint32_t)kSlotCap + (uint32_t)q;
    hid[up] = h;
    hid[lo] = h;
  }
}

__global__ void k_rowsort(int64_t N, const uint32_t* __restrict__ row_ptr,
                          uint32_t* __restrict__ col, DevCounters* __restrict__ cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  unsigned nd = 0;
  if (i < N) nd = sort_row(col + row_ptr[i], row_ptr[i + 1] - row_ptr[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nd = max(nd, __shfl_down_sync(0xffffffffu, nd, o));
  if ((threadIdx.x & 31) == 0 && nd) atomicMax(&cnt->max_degree_dip, nd);
}

}  // namespace

cudaError_t switch_run(const DevParams& P, const Table& t, const double* s, const float4* s32,
                       int precision, uint32_t epoch, SwitchBufs& b, DevCounters* cnt,
                       cudaStream_t st, int64_t* launches) {
  cudaError_t e = cudaMemsetAsync(b.indeg, 0, P.N * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(&cnt->sw_next, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  if (P.N <= 0) return cudaSuccess;
  // persistent grid: the resident blocks, at most one thread per site
  static int bps[2] = {0, 0};
  const int pi = precision == 1 ? 1 : 0;
  if (bps[pi] == 0) {
    e = pi ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps[pi], k_switch<1>, 256, 0)
           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps[pi], k_switch<0>, 256, 0);
    if (e != cudaSuccess) return e;
    if (bps[pi] < 1) bps[pi] = 1;
  }
  int64_t nb64 = (int64_t)bps[pi] * num_sms();
  if (nb64 > (P.N + 255) / 256) nb64 = (P.N + 255) / 256;
  const unsigned nb = (unsigned)nb64;
  if (precision == 1)
    k_switch<1><<<nb, 256, 0, st>>>(P, t.W, nullptr, t.disp, t.sw64, t.xyq, t.xy32, s, s32,
                                     epoch, t.m_nn[0], t.m_nn[1], b, cnt);
  else
    k_switch<0><<<nb, 256, 0, st>>>(P, t.W, t.Ebits, t.disp, t.sw64, t.xyq, t.xy32, s, s32,
                                     epoch, t.m_nn[0], t.m_nn[1], b, cnt);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t csr_scan(const DevParams& P, SwitchBufs& b, uint32_t* row_ptr, DevCounters* cnt,
                     cudaStream_t st, int64_t* launches) {
  k_degree<<<(unsigned)((P.N + 1 + 255) / 256), 256, 0, st>>>(P.N, b.hcnt, b.indeg, b.deg, cnt);
  ++*launches;
  return scan_excl_u32(b.deg, row_ptr, P.N + 1, b.scan_tmp,
                       reinterpret_cast<uint64_t*>(&cnt->nnz), st, launches);
}

cudaError_t csr_fill(const DevParams& P, const SwitchBufs& b, const uint32_t* row_ptr,
                     uint32_t* col, uint32_t* hid, bool has_overflow, bool sort_rows,
                     DevCounters* cnt, cudaStream_t st, int64_t* launches) {
  cudaError_t e = cudaMemsetAsync(b.lcur, 0, P.N * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  const unsigned nb = (unsigned)((P.N + 255) / 256);
  k_fill<<<nb, 256, 0, st>>>(P.N, b.hslot, b.hcnt, b.indeg, row_ptr, b.lcur, col, hid);
  ++*launches;
  if (has_overflow) {
    unsigned long long n = 0;
    e = cudaMemcpyAsync(&n, &cnt->ovf_n, sizeof(n), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    if (n > b.ovf_cap) n = b.ovf_cap;
    e = cudaMemsetAsync(b.ocur, 0, P.N * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    if (n > 0) {
      k_fill_ovf<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, (uint32_t)P.N, b.ovf, b.indeg,
                                                              row_ptr, b.lcur, b.ocur, col, hid);
      ++*launches;
    }
  }
  if (sort_rows) {  // (the half-edge ids are not moved: callers that keep them leave rows unsorted)
    if (hid) return cudaErrorInvalidValue;
    k_rowsort<<<nb, 256, 0, st>>>(P.N, row_ptr, col, cnt);
    ++*launches;
  }
  return cudaGetLastError();
}

cudaError_t csr_sorted_copy(const DevParams& P, const uint32_t* row_ptr, const uint32_t* col,
                            uint32_t* out, uint64_t nnz, DevCounters* cnt, cudaStream_t st,
                            int64_t* launches) {
  cudaError_t e = cudaMemcpyAsync(out, col, nnz * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  k_rowsort<<<(unsigned)((P.N + 255) / 256), 256, 0, st>>>(P.N, row_ptr, out, cnt);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace sco
