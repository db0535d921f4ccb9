// kw_low.cuh -- the first levels of the Kuhn-Wattenhofer colouring (Sec. 2.3.3) inside one
// thread block.
//
// At level p the groups are runs of g 2^p consecutive vertices (v / (g 2^p)), and a vertex only
// looks at same-group neighbours.  So while g 2^p0 <= kLowMaxGroup, a level-p0 group goes
// through levels 1..p0 without any edge that leaves it: one block takes the group alone.  Its
// internal edges are staged in shared memory once, each tagged with the level at which its two
// ends join one group (or read from the rows when they do not fit).  Every level first builds,
// in parallel, a record per right-half vertex (the colours of its left-half neighbours, final
// at this level, and its right-half neighbours of larger previous colour), stored in bucket
// order, then runs the plain colour reduction (2) of Sec. 2.3.2 over the buckets of equal
// previous colour, from the largest down, one __syncthreads apart: a bucket step reads a
// record and the states of its listed neighbours only.  By the
// bucket-order lemma of the grid-wide colouring kernels this gives the colours and per-level
// rounds of the synchronous rounds of (2)'.  The grid-wide kernels then start at level p0 + 1.
#pragma once

#include <cstdint>

#include "batch.h"
#include "grid_dev.cuh"
#include "kw_dev.cuh"

namespace sco {
namespace {

constexpr uint32_t kLowMaxGroup = 4096;  // vertices of one block-local group
constexpr uint32_t kLowMaxPal = 64;      // palettes g <= 64: colour sets are 64-bit masks
constexpr int kLowThreads = 256;

// Levels taken block-locally for a lattice of palette g and M levels with groups of at most
// gmax <= kLowMaxGroup vertices (0: none; gmax = 0 turns the block-local levels off).
__host__ __device__ __forceinline__ unsigned kw_low_levels(uint32_t g, unsigned M,
                                                          uint32_t gmax) {
  if (g == 0 || g > kLowMaxPal || gmax > kLowMaxGroup) return 0;
  unsigned p = 0;
  while (p < M && ((unsigned long long)g << (p + 1)) <= gmax) ++p;
  return p;
}

struct KwLowView {
  int R;                        // lattices (1 for a single lattice)
  const uint32_t* site_start;   // R + 1 first vertex of each lattice
  const RepPlan* plan;          // R: g, levels, magic
  const uint32_t* row_ptr;      // global entry offsets; col entries lattice-local
  const uint32_t* col;
  unsigned long long* word;     // packed (level, round, colour), global vertex index
  uint8_t* col8;                // colour (low byte), global vertex index
  DevCounters* cnt;             // R: lev_rounds
  const int* halt;              // optional: nonzero on entry -> return at once
  uint32_t gmax;                // group-size cap of kw_low_levels
  uint32_t gcap;                // >= every group size g 2^p0, <= gmax, even
  uint32_t ecap;                // internal edges staged per group (0: rows at every level)
};

// Dynamic shared memory of k_kw_low: bucket records (16 bytes per right-half vertex), site
// bases and group prefix (R + 1 each), bucket starts and cursors, per-level rounds, two words
// of block state (u32); vertex states, first internal edges and edges (u16); internal degrees
// (u8).
inline size_t kw_low_smem(int R, uint32_t gcap, uint32_t ecap) {
  return (size_t)(gcap / 2 + 1) * 16 +
         (size_t)(2 * (R + 1) + (kLowMaxPal + 1) + kLowMaxPal + 32 + 2) * 4 +
         (size_t)(gcap + gcap + ecap) * 2 + gcap;
}

// Largest edge capacity (<= 2^16 - 1) that keeps `blocks` blocks of k_kw_low on one SM.
inline uint32_t kw_low_ecap(int R, uint32_t gcap, int blocks, size_t smem_per_sm) {
  const size_t per = smem_per_sm / (size_t)blocks;
  const size_t reserve = 1024 + 64;  // per-block memory the runtime keeps, static variables
  const size_t fixed = kw_low_smem(R, gcap, 0);
  if (per < fixed + reserve) return 0;
  const size_t e = (per - fixed - reserve) / 2;
  return (uint32_t)(e > 65535 ? 65535 : e);
}

// Blocks per SM and edge capacity: the most blocks whose capacity still holds five internal
// edges per vertex (a denser group falls back to reading its rows).
inline void kw_low_shape(int R, uint32_t gcap, size_t smem_per_sm, size_t smem_per_block,
                         int* blocks, uint32_t* ecap) {
  int b = 8;
  uint32_t e = kw_low_ecap(R, gcap, b, smem_per_sm);
  while (b > 1 && e < 5 * gcap) e = kw_low_ecap(R, gcap, --b, smem_per_sm);
  while (kw_low_smem(R, gcap, e) > smem_per_block && e > 0) e = e > 1024 ? e - 1024 : 0;
  *blocks = b;
  *ecap = e;
}

// l / g for l < kLowMaxGroup, g <= kLowMaxPal: one multiply-high with m = floor(2^32 / g) + 1
// (exact there: the error l (m g - 2^32) / 2^32 stays below 1 / g); g = 1 passes m = 0.
__host__ __device__ __forceinline__ uint32_t low_magic(uint32_t g) {
  return g > 1 ? (uint32_t)(0xFFFFFFFFull / g + 1ull) : 0u;
}
__device__ __forceinline__ uint32_t low_div(uint32_t l, uint32_t m) {
  return m ? __umulhi(l, m) : l;
}

// Level at which level-0 groups bx and by first lie in one group (0: the same group).
__device__ __forceinline__ uint32_t low_join(uint32_t bx, uint32_t by) {
  return 32u - (uint32_t)__clz((int)(bx ^ by));
}

// An internal edge in shared memory: group-local neighbour (12 bits) | join level << 12.
constexpr uint32_t kLowY = 0x0FFFu;
// Vertex state (u16): colour (6 bits) | round at its last recolouring << 6 (7 bits) | done at
// the current level << 13.
constexpr uint32_t kLowDone = 1u << 13;
// Bucket record (uint4): {left-half colour mask lo, hi, v | n << 12 | y0 << 16, y1 | y2 << 16}
// with n <= kLowRecList listed larger right-half neighbours, or kLowRecMore (scan instead).
constexpr uint32_t kLowRecList = 3;
constexpr uint32_t kLowRecMore = 7;

__device__ __forceinline__ void low_prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Neighbours of right-half vertex v at level p through its staged edges (or its row): calls
// f(y, lv) for every same-group one (join level lv <= p).
template <class F>
__device__ __forceinline__ void low_for_nbrs(bool staged, uint32_t v, uint32_t bx,
                                             const uint16_t* es, const uint8_t* ek,
                                             const uint16_t* edges,
                                             const uint32_t* __restrict__ rowp,
                                             const uint32_t* __restrict__ col, uint32_t v0,
                                             uint32_t n, uint32_t m32, unsigned p, F&& f) {
  if (staged) {
    const uint32_t q1 = es[v] + ek[v];
    for (uint32_t q = es[v]; q < q1; ++q) {
      const uint32_t ev = edges[q], lv = ev >> 12;
      if (lv <= p) f(ev & kLowY, lv);
    }
  } else {
    const uint32_t q1 = rowp[v + 1];
    for (uint32_t q = rowp[v]; q < q1; ++q) {
      const uint32_t y = (col[q] & kIndexMask) - v0;
      if (y >= n) continue;
      const uint32_t lv = low_join(bx, low_div(y, m32));
      if (lv <= p) f(y, lv);
    }
  }
}

// Levels 1..kw_low_levels(g, M, gmax) of every lattice, one level-p0 group per block at a time.
// Overwrites the words of those lattices (after the initial colours were written) and raises
// lev_rounds[1..p0].
__global__ void __launch_bounds__(kLowThreads, 4) k_kw_low(const KwLowView V) {
  __shared__ int s_halt;
  if (threadIdx.x == 0) s_halt = V.halt ? ld_status(V.halt) : 0;
  __syncthreads();
  if (s_halt) return;
  extern __shared__ uint4 lsm4[];
  const int R = V.R;
  const uint32_t gcap = V.gcap;
  uint4* rec = lsm4;                                  // gcap / 2 + 1 bucket records
  uint32_t* sbase = reinterpret_cast<uint32_t*>(rec + gcap / 2 + 1);  // R + 1
  uint32_t* gp = sbase + R + 1;           // R + 1 group prefix
  uint32_t* bst = gp + R + 1;             // kLowMaxPal + 1 bucket starts
  uint32_t* cur = bst + kLowMaxPal + 1;   // kLowMaxPal bucket cursors
  uint32_t* rl = cur + kLowMaxPal;        // 32 deepest round per level (this group)
  uint32_t* blk = rl + 32;                // [0] edge cursor, [1] overflow
  uint16_t* st = reinterpret_cast<uint16_t*>(blk + 2);  // gcap vertex states
  uint16_t* es = st + gcap;               // gcap first internal edge
  uint16_t* edges = es + gcap;            // ecap internal edges
  uint8_t* ek = reinterpret_cast<uint8_t*>(edges + V.ecap);  // gcap internal degrees
  const uint32_t T = blockDim.x, tid = threadIdx.x;
  const int lane = (int)(tid & 31);
  for (int r = tid; r < R; r += T) {
    const RepPlan pl = V.plan[r];
    const uint32_t b0 = V.site_start[r], N = V.site_start[r + 1] - b0;
    const unsigned low = kw_low_levels(pl.g, pl.levels, V.gmax);
    const uint32_t G = pl.g << low;
    sbase[r] = b0;
    gp[r] = low ? (N + G - 1) / G : 0u;
  }
  if (tid == 0) sbase[R] = V.site_start[R];
  __syncthreads();
  if (tid < 32) {  // exclusive prefix of the group counts, 32 lattices at a time
    uint32_t run = 0;
    for (int r0 = 0; r0 < R; r0 += 32) {
      const int r = r0 + lane;
      const uint32_t v = r < R ? gp[r] : 0u;
      uint32_t x = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
      }
      if (r < R) gp[r] = run + x - v;
      run += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) gp[R] = run;
  }
  __syncthreads();
  const uint32_t total = gp[R];
  // group gi of lattice r: first vertex, size
  auto group_of = [&](uint32_t gi, int& r, uint32_t& v0, uint32_t& n) {
    r = find_le(gp, R, gi);
    const RepPlan pl = V.plan[r];
    const uint32_t G = pl.g << kw_low_levels(pl.g, pl.levels, V.gmax);
    const uint32_t N = sbase[r + 1] - sbase[r];
    v0 = (gi - gp[r]) * G;
    n = min(G, N - v0);
  };
  for (uint32_t gi = blockIdx.x; gi < total; gi += gridDim.x) {
    int r;
    uint32_t v0, n;
    group_of(gi, r, v0, n);
    const RepPlan pl = V.plan[r];
    const uint32_t g = pl.g;
    const uint32_t m32 = low_magic(g);
    const unsigned low = kw_low_levels(g, pl.levels, V.gmax);
    const uint32_t base = sbase[r];
    const uint32_t* rowp = V.row_ptr + base + v0;
    if (tid < 32) rl[tid] = 0;
    if (tid == 0) {
      blk[0] = 0;
      blk[1] = 0;
    }
    __syncthreads();
    // initial colours (l mod g: v0 is a multiple of g) and the internal edges: each vertex
    // counts them (sixteen loads in flight), takes a slice of the edge array (one atomic per
    // warp) and writes them from the row again, tagged with their join level
    for (uint32_t l0 = 0; l0 < n; l0 += T) {
      const uint32_t l = l0 + tid;
      const bool on = l < n;
      uint32_t bx = 0, b = 0, e = 0, k = 0;
      if (on) {
        bx = low_div(l, m32);
        st[l] = (uint16_t)(l - bx * g);
        b = rowp[l];
        e = rowp[l + 1];
      }
      for (uint32_t a0 = b; a0 < e; a0 += 16) {
        uint32_t y[16];
#pragma unroll
        for (int a = 0; a < 16; ++a)
          y[a] = a0 + a < e ? (V.col[a0 + a] & kIndexMask) - v0 : 0xFFFFFFFFu;
#pragma unroll
        for (int a = 0; a < 16; ++a) k += y[a] < n;
      }
      uint32_t x = k;  // warp-inclusive scan of the counts
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
      }
      uint32_t wb = 0;
      if (lane == 31) wb = atomicAdd(&blk[0], x);
      wb = __shfl_sync(0xffffffffu, wb, 31);
      const uint32_t pos = wb + x - k;
      if (!on) continue;
      ek[l] = (uint8_t)k;
      if (pos + k > V.ecap) {
        blk[1] = 1;
        continue;
      }
      es[l] = (uint16_t)pos;
      uint32_t w = pos;
      for (uint32_t a0 = b; a0 < e; a0 += 16) {
        uint32_t y[16];
#pragma unroll
        for (int a = 0; a < 16; ++a)
          y[a] = a0 + a < e ? (V.col[a0 + a] & kIndexMask) - v0 : 0xFFFFFFFFu;
#pragma unroll
        for (int a = 0; a < 16; ++a)
          if (y[a] < n) edges[w++] = (uint16_t)(y[a] | (low_join(bx, low_div(y[a], m32)) << 12));
      }
    }
    // the rows of this block's next group, into L2 while this one runs its levels
    if (gi + gridDim.x < total) {
      int r2;
      uint32_t v2, n2;
      group_of(gi + gridDim.x, r2, v2, n2);
      const uint32_t* rp2 = V.row_ptr + sbase[r2] + v2;
      for (uint32_t q = tid * 32; q <= n2; q += T * 32) low_prefetch_l2(rp2 + q);
      const uint32_t c0 = rp2[0], c1 = rp2[n2];
      for (uint32_t q = c0 + tid * 32; q < c1; q += T * 32) low_prefetch_l2(V.col + q);
    }
    __syncthreads();
    const bool staged = blk[1] == 0;
    for (unsigned p = 1; p <= low; ++p) {
      // right half of level p: runs of half = g 2^(p-1) vertices starting at odd multiples of
      // half; slot s lies in run k = s / half, vertex s + (k + 1) half
      const uint32_t half = g << (p - 1);
      const uint32_t rem = n % (2 * half);
      const uint32_t nr = n / (2 * half) * half + (rem > half ? rem - half : 0u);
      auto right_vertex = [&](uint32_t sl) {
        return sl + ((low_div(sl, m32) >> (p - 1)) + 1) * half;
      };
      __syncthreads();  // every thread is past the previous level's bucket starts
      if (tid <= kLowMaxPal) bst[tid] = 0;
      if (tid < kLowMaxPal) cur[tid] = 0;
      __syncthreads();
      // right half: not done yet, bucket sizes by previous colour
      for (uint32_t sl = tid; sl < nr; sl += T) {
        const uint32_t l = right_vertex(sl);
        const uint32_t s = st[l] & ~kLowDone;
        st[l] = (uint16_t)s;
        atomicAdd(&bst[s & 63u], 1u);
      }
      __syncthreads();
      if (tid < 32) {
        const uint32_t i0 = 2 * tid, i1 = i0 + 1;
        const uint32_t a0 = i0 < g ? bst[i0] : 0u, a1 = i1 < g ? bst[i1] : 0u;
        uint32_t x = a0 + a1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
          if ((int)tid >= o) x += y;
        }
        const uint32_t ex = x - a0 - a1;
        if (i0 < g) bst[i0] = ex;
        if (i1 < g) bst[i1] = ex + a0;
        if (tid == 31) bst[g] = x;
      }
      __syncthreads();
      // records, in bucket order: every colour still holds its value from level p - 1
      for (uint32_t sl = tid; sl < nr; sl += T) {
        const uint32_t l = right_vertex(sl), bx = low_div(l, m32);
        const uint32_t c = st[l] & 63u;
        unsigned long long mask = 0;
        uint32_t m = 0, ys[kLowRecList] = {0, 0, 0};
        low_for_nbrs(staged, l, bx, es, ek, edges, rowp, V.col, v0, n, m32, p,
                     [&](uint32_t y, uint32_t lv) {
                       const uint32_t cy = st[y] & 63u;
                       if (lv == p) {
                         mask |= 1ull << cy;
                       } else if (cy > c) {
                         if (m < kLowRecList) ys[m] = y;
                         ++m;
                       }
                     });
        const uint32_t nn = m <= kLowRecList ? m : kLowRecMore;
        rec[bst[c] + atomicAdd(&cur[c], 1u)] =
            make_uint4((uint32_t)mask, (uint32_t)(mask >> 32), l | (nn << 12) | (ys[0] << 16),
                       ys[1] | (ys[2] << 16));
      }
      __syncthreads();
      // buckets from the largest previous colour down, one vertex per thread; a thread's record
      // of the next bucket (and that bucket's bounds) are loaded before this bucket's barrier
      uint32_t rmax = 0;
      uint32_t s0 = bst[g - 1], s1 = bst[g];
      uint4 qn = make_uint4(0, 0, 0, 0);
      if (tid < s1 - s0) qn = rec[s0 + tid];
      for (int c = (int)g - 1; c >= 0; --c) {
        const uint32_t b0 = s0, nb = s1 - s0;
        const uint4 q0 = qn;
        if (c > 0) {
          s1 = s0;
          s0 = bst[c - 1];
          if (tid < s1 - s0) qn = rec[s0 + tid];
        }
        if (nb == 0) continue;
        for (uint32_t j = tid; j < nb; j += T) {
          const uint4 q = j == tid ? q0 : rec[b0 + j];
          const uint32_t v = q.z & kLowY, nn = (q.z >> 12) & 7u;
          unsigned long long mask = q.x | ((unsigned long long)q.y << 32);
          uint32_t rv = 0;
          auto take = [&](uint32_t sy) {
            mask |= 1ull << (sy & 63u);
            rv = max(rv, (sy >> 6) & 0x7Fu);
          };
          if (nn != kLowRecMore) {
            const uint32_t y0 = q.z >> 16, y1 = q.w & 0xFFFFu, y2 = q.w >> 16;
            if (nn > 0) take(st[y0]);
            if (nn > 1) take(st[y1]);
            if (nn > 2) take(st[y2]);
          } else {  // larger right-half neighbours are the ones done at this level
            low_for_nbrs(staged, v, low_div(v, m32), es, ek, edges, rowp, V.col, v0, n, m32, p,
                         [&](uint32_t y, uint32_t lv) {
                           const uint32_t sy = st[y];
                           if (lv < p && (sy & kLowDone)) take(sy);
                         });
          }
          const uint32_t cn = (uint32_t)(__ffsll((long long)~mask) - 1);
          st[v] = (uint16_t)(cn | ((rv + 1) << 6) | kLowDone);
          rmax = max(rmax, rv + 1);
        }
        __syncthreads();
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) rmax = max(rmax, __shfl_down_sync(0xffffffffu, rmax, o));
      if (lane == 0 && rmax) atomicMax(&rl[p], rmax);
    }
    __syncthreads();
    // words: colour, round at the last recolouring, and that level (the highest of the
    // first p0 levels at which the vertex was in a right half; 0 if none)
    unsigned long long* word = V.word + base + v0;
    uint8_t* col8 = V.col8 + base + v0;
    for (uint32_t l = tid; l < n; l += T) {
      const uint32_t s = st[l];
      const uint32_t bits = low_div(l, m32) & ((1u << low) - 1u);
      const uint32_t tag = bits ? 32u - (uint32_t)__clz((int)bits) : 0u;
      word[l] = pack(tag, tag ? (s >> 6) & 0x7Fu : 0u, s & 63u);
      col8[l] = (uint8_t)(s & 63u);
    }
    if (tid >= 1 && tid <= low && rl[tid]) atomicMax(&V.cnt[r].lev_rounds[tid & 31], rl[tid]);
    __syncthreads();  // shared memory is reused by the next group
  }
}

}  // namespace
}  // namespace sco
