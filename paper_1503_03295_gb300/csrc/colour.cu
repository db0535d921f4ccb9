// colour.cu -- step (2) of Fig. 1: Kuhn-Wattenhofer colouring of the switched graph
// (Sec. 2.3.3) with the modified colour reduction (2)' of Sec. 2.3.2, and the colour
// classes (sites grouped by colour) used by the colour-class sweep.
//
// Vertex v starts with colour v; with g = Delta + 1 its level-0 group is v / g and its
// colour inside the group v mod g.  At level p the groups are v / (g 2^p); the right half
// of every group (colours shifted to [g, 2g)) is reduced back into [0, g).
//
// Schedule.  In a synchronous round of (2)' a right-half vertex recolours once every
// same-group neighbour with a larger colour has left [g, 2g); its new colour is the smallest
// colour not held by a same-group neighbour, and at that moment the neighbours that matter
// (colour < g) are exactly the left half and the right-half neighbours with a larger
// previous colour, all of them final.  The result therefore does not depend on the order
// in which ready vertices are processed, and the synchronous round of a vertex is one more
// than the largest round among those larger neighbours.  Each level runs as one persistent
// cooperative kernel in which every thread repeatedly visits its own vertices and
// recolours those whose larger neighbours are done: no grid-wide barrier between rounds,
// same colours as the synchronous rounds, and t_R recovered from the per-vertex rounds.
#include <cstdint>

#include "sco_internal.h"

namespace sco {

namespace {

constexpr int kStatusTimeout = 4;
constexpr unsigned long long kColMask = 0xFFFFFFFFull;

// word = tag (level) << 48 | round << 32 | colour
__device__ __forceinline__ unsigned long long pack(unsigned p, unsigned r, unsigned c) {
  return ((unsigned long long)p << 48) | ((unsigned long long)r << 32) | c;
}
__device__ __forceinline__ unsigned tag_of(unsigned long long w) { return (unsigned)(w >> 48); }
__device__ __forceinline__ unsigned rnd_of(unsigned long long w) {
  return (unsigned)(w >> 32) & 0xFFFFu;
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_status(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__global__ void k_kw_init(int64_t N, uint32_t g, unsigned long long* __restrict__ word) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v < N) word[v] = pack(0, 0, (unsigned)(v % g));
}

// floor(u / g) for 32-bit u and g by one 64-bit high multiply with M = floor((2^64-1)/g) + 1
// (Lemire, Kaser and Kurz, "Faster remainder by direct computation", 2019).
__device__ __forceinline__ uint32_t fdiv(uint32_t u, unsigned long long M) {
  return (uint32_t)__umul64hi(M, (unsigned long long)u);
}

// Smallest colour in [0, g) not held by a ready same-group neighbour (mex <= degree).
__device__ __noinline__ unsigned mex_slow(uint32_t v, unsigned p, unsigned long long M,
                                          const uint32_t* __restrict__ row_ptr,
                                          const uint32_t* __restrict__ col,
                                          const unsigned long long* word) {
  const uint32_t b = row_ptr[v], e = row_ptr[v + 1];
  const uint32_t grp = fdiv(v, M) >> p;
  for (unsigned c = 0;; ++c) {
    bool used = false;
    for (uint32_t q = b; q < e && !used; ++q) {
      const uint32_t u = col[q] & kIndexMask;
      const uint32_t gu = fdiv(u, M);
      if ((gu >> p) != grp) continue;
      const unsigned long long wu = ld_relaxed(&word[u]);
      if (((gu >> (p - 1)) & 1u) && tag_of(wu) != p) continue;
      used = (unsigned)(wu & kColMask) == c;
    }
    if (!used) return c;
  }
}

__global__ void __launch_bounds__(256) k_kw_level(uint32_t N, uint32_t g, unsigned long long M,
                                                  unsigned p, const uint32_t* __restrict__ row_ptr,
                                                  const uint32_t* __restrict__ col,
                                                  unsigned long long* word,
                                                  DevCounters* __restrict__ cnt,
                                                  unsigned long long ns_limit) {
  const unsigned long long t_start = global_ns();
  const uint32_t half = g << (p - 1);
  const uint32_t ngroups = (uint32_t)(((unsigned long long)N + ((unsigned long long)g << p) - 1) /
                                      ((unsigned long long)g << p));
  const uint32_t R = ngroups * half;  // right-half slots (some beyond N)
  const uint32_t nth = gridDim.x * blockDim.x;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned rmax = 0;
  bool pending = true;
  for (unsigned long long pass = 0; pending; ++pass) {
    pending = false;
    for (uint32_t r = tid; r < R; r += nth) {
      const uint32_t k = fdiv(r, M) >> (p - 1);  // right half number k -> group k
      const uint32_t v = (2 * k + 1) * half + (r - k * half);
      if (v >= N) continue;
      const unsigned long long wv = ld_relaxed(&word[v]);
      if (tag_of(wv) == p) continue;
      const uint32_t cv = (uint32_t)(wv & kColMask);
      const uint32_t grp = k;  // v / (g 2^p)
      const uint32_t b = row_ptr[v], e = row_ptr[v + 1];
      unsigned long long used[4] = {0, 0, 0, 0};  // colours < 256 (mex <= degree)
      bool blocked = false;
      unsigned rv = 0;
      for (uint32_t q = b; q < e; ++q) {
        const uint32_t u = col[q] & kIndexMask;
        const uint32_t gu = fdiv(u, M);
        if ((gu >> p) != grp) continue;
        const unsigned long long wu = ld_relaxed(&word[u]);
        const uint32_t cu = (uint32_t)(wu & kColMask);
        const bool right = (gu >> (p - 1)) & 1u;
        if (right && tag_of(wu) != p) {
          if (cu > cv) {  // larger same-group neighbour still in [g, 2g): wait
            blocked = true;
            break;
          }
          continue;  // smaller one: its colour is >= g for now and it waits for v
        }
        if (right) rv = max(rv, rnd_of(wu));
        if (cu < 256) used[cu >> 6] |= 1ull << (cu & 63);
      }
      if (blocked) {
        pending = true;
        continue;
      }
      unsigned c = 0;
      if (e - b < 256) {
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          if (~used[w]) {
            c = 64 * w + __ffsll((long long)~used[w]) - 1;
            break;
          }
        }
      } else {
        c = mex_slow(v, p, M, row_ptr, col, word);
      }
      rmax = max(rmax, rv + 1);
      st_relaxed(&word[v], pack(p, rv + 1, c));
    }
    // bounded wait: give up (status SCO_ETIMEOUT) after ns_limit of wall time or when another
    // thread already failed
    if (pending && ((pass & 15) == 15) &&
        (global_ns() - t_start > ns_limit || ld_status(&cnt->status) != 0)) {
      atomicCAS(&cnt->status, 0, kStatusTimeout);
      break;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rmax = max(rmax, __shfl_down_sync(0xffffffffu, rmax, o));
  if ((threadIdx.x & 31) == 0 && rmax) atomicMax(&cnt->lev_rounds[p & 31], rmax);
}

__global__ void k_kw_final(int64_t N, unsigned levels, uint32_t g, int variant,
                           const unsigned long long* __restrict__ word,
                           uint32_t* __restrict__ colour, DevCounters* __restrict__ cnt) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v < N) colour[v] = (uint32_t)(word[v] & kColMask);
  if (v == 0) {
    unsigned t = 0;
    for (unsigned p = 1; p <= levels; ++p) t += cnt->lev_rounds[p & 31];
    // plain BCR (2) spends exactly g rounds per level on the same colouring
    cnt->kw_rounds = variant == 1 ? g * levels : t;
    cnt->levels = levels;
  }
}

// ---- colour classes --------------------------------------------------------------------
__global__ void k_hist(int64_t N, const uint32_t* __restrict__ colour, uint32_t* __restrict__ hist) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool ok = v < N;
  const uint32_t c = ok ? colour[v] : 0xFFFFFFFFu;
  const unsigned mask = __match_any_sync(0xffffffffu, c);
  const int lane = threadIdx.x & 31;
  if (ok && lane == __ffs(mask) - 1) atomicAdd(&hist[c], (uint32_t)__popc(mask));
}

__global__ void k_nonempty(uint32_t g, const uint32_t* __restrict__ hist,
                           DevCounters* __restrict__ cnt) {
  unsigned n = 0;
  for (uint32_t c = threadIdx.x; c < g; c += blockDim.x) n += hist[c] > 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0 && n) atomicAdd(&cnt->n_colours, n);
}

// Sites of one colour keep ascending order inside a warp; warps claim their ranges with
// one atomic per colour and warp.  The order inside a class does not affect the results
// (sites of one colour never interact).
__global__ void k_scatter(int64_t N, const uint32_t* __restrict__ colour,
                          const uint32_t* __restrict__ off, uint32_t* __restrict__ cursor,
                          uint32_t* __restrict__ perm) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool ok = v < N;
  const uint32_t c = ok ? colour[v] : 0xFFFFFFFFu;
  const unsigned mask = __match_any_sync(0xffffffffu, c);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  uint32_t base = 0;
  if (ok && lane == leader) base = atomicAdd(&cursor[c], (uint32_t)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  if (ok) perm[off[c] + base + __popc(mask & ((1u << lane) - 1u))] = (uint32_t)v;
}

}  // namespace

cudaError_t kw_run(const DevParams& P, const uint32_t* row_ptr, const uint32_t* col,
                   uint32_t g, int variant, ColourBufs& b, DevCounters* cnt, cudaStream_t st,
                   int64_t* launches) {
  const int64_t N = P.N;
  const int64_t G = (N + g - 1) / g;
  unsigned M = 0;  // levels (N < 2^30 keeps every index below 2^32)
  while (((int64_t)1 << M) < G) ++M;
  cudaError_t e = cudaMemsetAsync(cnt->lev_rounds, 0, sizeof(cnt->lev_rounds), st);
  if (e != cudaSuccess) return e;
  const unsigned nb = (unsigned)((N + 255) / 256);
  k_kw_init<<<nb, 256, 0, st>>>(N, g, b.word);
  ++*launches;
  static int blocks_per_sm = 0;
  if (blocks_per_sm == 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_kw_level, 256, 0);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  const int64_t want = (N / 2 + 255) / 256;
  int64_t grid = (int64_t)blocks_per_sm * num_sms();
  if (want < grid) grid = want > 0 ? want : 1;
  const unsigned long long ns_limit = 2000000000ull;  // 2 s per level
  unsigned long long magic = 0xFFFFFFFFFFFFFFFFull / g + 1ull;
  for (unsigned p = 1; p <= M; ++p) {
    uint32_t Nn = (uint32_t)N;
    uint32_t gg = g;
    unsigned pp = p;
    unsigned long long lim = ns_limit;
    void* args[] = {(void*)&Nn, (void*)&gg, (void*)&magic, (void*)&pp, (void*)&row_ptr,
                    (void*)&col, (void*)&b.word, (void*)&cnt, (void*)&lim};
    e = cudaLaunchCooperativeKernel((const void*)k_kw_level, dim3((unsigned)grid), dim3(256),
                                    args, 0, st);
    if (e != cudaSuccess) return e;
    ++*launches;
  }
  k_kw_final<<<nb, 256, 0, st>>>(N, M, g, variant, b.word, b.colour, cnt);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t bucket_run(const DevParams& P, uint32_t g, ColourBufs& b, DevCounters* cnt,
                       cudaStream_t st, int64_t* launches) {
  const int64_t N = P.N;
  cudaError_t e = cudaMemsetAsync(b.hist, 0, (g + 1) * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.cursor, 0, g * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(&cnt->n_colours, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const unsigned nb = (unsigned)((N + 255) / 256);
  k_hist<<<nb, 256, 0, st>>>(N, b.colour, b.hist);
  ++*launches;
  k_nonempty<<<1, 1024, 0, st>>>(g, b.hist, cnt);
  ++*launches;
  e = scan_excl_u32(b.hist, b.off, (int64_t)g + 1, b.scan_tmp, nullptr, st, launches);
  if (e != cudaSuccess) return e;
  k_scatter<<<nb, 256, 0, st>>>(N, b.colour, b.off, b.cursor, b.perm);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace sco
