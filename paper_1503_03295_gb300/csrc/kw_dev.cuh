// kw_dev.cuh -- per-vertex step of the Kuhn-Wattenhofer colouring (Sec. 2.3.3) with the
// modified colour reduction (2)' of Sec. 2.3.2, shared by the single-lattice and batched
// colouring kernels.
//
// Vertex v starts with colour v; with g = Delta + 1 its level-0 group is v / g and its
// colour inside the group v mod g.  At level p the groups are v / (g 2^p); the right half
// of every group (colours shifted to [g, 2g)) is reduced back into [0, g).  A right-half
// vertex recolours once every same-group neighbour with a larger colour has done so; its new
// colour is the smallest one not held by a same-group neighbour that is final at that
// moment, and its synchronous round is one more than the largest round among those larger
// neighbours.  The result does not depend on the order in which ready vertices go.
#pragma once

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
// One-byte colour copies (palettes <= 64): 32 sites per sector for the neighbour gathers.
__device__ __forceinline__ uint32_t ld_relaxed_u8(const uint8_t* p) {
  unsigned short v;
  asm volatile("ld.relaxed.gpu.global.u8 %0, [%1];" : "=h"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u8(uint8_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u8 [%0], %1;" ::"l"(p), "h"((unsigned short)v) : "memory");
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

// How often a bounded wait reads the clock: every 256th spin (every 16th pass) for the normal
// limits of seconds, every spin (pass) for limits below 1 ms, so that a short limit is honoured
// within one spin.  Returns the mask tested against the spin (or pass) counter.
constexpr unsigned long long kShortWaitNs = 1000000ull;
__device__ __forceinline__ unsigned wait_spin_mask(unsigned long long ns_limit) {
  return ns_limit < kShortWaitNs ? 0u : 255u;
}
__device__ __forceinline__ unsigned wait_pass_mask(unsigned long long ns_limit) {
  return ns_limit < kShortWaitNs ? 0u : 15u;
}

// floor(u / g) through the multiplier of g (see div_by_magic).
__device__ __forceinline__ uint32_t fdiv(uint32_t u, unsigned long long M) {
  return div_by_magic(u, M);
}

// Smallest colour in [0, g) not held by a ready same-group neighbour (mex <= degree).
__device__ __noinline__ unsigned mex_slow(uint32_t v, unsigned p, unsigned long long M,
                                          const uint32_t* __restrict__ col,
                                          const unsigned long long* word, uint32_t b,
                                          uint32_t e) {
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

// One KW level.  Thread t owns the right-half slots r = t + k * nthreads.  It passes over
// its unfinished vertices again and again: a vertex whose recorded blocker (a larger
// same-group right-half neighbour not yet recoloured at this level) is still unfinished
// costs one load; otherwise its row is scanned, and it either records the unfinished
// larger neighbour of smallest colour (the one likely to finish last) or takes the
// smallest colour not held by a finished same-group neighbour.  Nothing ever blocks a
// thread, so with every thread resident the unfinished vertex of largest colour in each
// group always progresses.
constexpr uint32_t kNone = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t kw_vertex(uint32_t r, uint32_t half, unsigned p,
                                              unsigned long long M) {
  const uint32_t k = fdiv(r, M) >> (p - 1);  // right half number k, in group k
  return (2 * k + 1) * half + (r - k * half);
}

// Returns kNone once v is recoloured, else the index of the neighbour to wait for.
__device__ __noinline__ uint32_t kw_attempt(uint32_t v, uint32_t cv, unsigned p,
                                               unsigned long long M,
                                               const uint32_t* __restrict__ row_ptr,
                                               const uint32_t* __restrict__ col,
                                               unsigned long long* word, unsigned& rmax) {
  const uint32_t grp = fdiv(v, M) >> p;
  const uint32_t b = row_ptr[v], e = row_ptr[v + 1];
  unsigned long long used[4] = {0, 0, 0, 0};  // colours < 256 (mex <= degree)
  unsigned rv = 0;
  uint32_t wait_u = kNone, wait_c = 0xFFFFFFFFu;
  // the row in chunks of 8: indices, then the words of the same-group ones, back to back
  for (uint32_t q0 = b; q0 < e; q0 += 8) {
    uint32_t uu[8];
    unsigned long long ww[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) uu[a] = q0 + a < e ? (col[q0 + a] & kIndexMask) : kNone;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      ww[a] = 0;
      if (uu[a] != kNone && (fdiv(uu[a], M) >> p) == grp) ww[a] = ld_relaxed(&word[uu[a]]);
      else uu[a] = kNone;
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      if (uu[a] == kNone) continue;
      const unsigned long long wu = ww[a];
      const uint32_t cu = (uint32_t)(wu & kColMask);
      const bool right = (fdiv(uu[a], M) >> (p - 1)) & 1u;
      if (right && tag_of(wu) != p) {
        // larger: must finish first; smaller: its colour is >= g for now and it waits for v
        if (cu > cv && cu < wait_c) {
          wait_c = cu;
          wait_u = uu[a];
        }
        continue;
      }
      if (right) rv = max(rv, rnd_of(wu));
      if (cu < 256) used[cu >> 6] |= 1ull << (cu & 63);
    }
  }
  if (wait_u != kNone) return wait_u;
  unsigned cn = 0;
  if (e - b < 256) {
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      if (~used[w]) {
        cn = 64 * w + __ffsll((long long)~used[w]) - 1;
        break;
      }
    }
  } else {
    cn = mex_slow(v, p, M, col, word, b, e);
  }
  rmax = max(rmax, rv + 1);
  st_relaxed(&word[v], pack(p, rv + 1, cn));
  return kNone;
}


// Pending vertices (bits of pend) that may try now: those with no recorded blocker, and those
// whose blocker has been recoloured at level p.  The blockers' words are loaded eight at a
// time, back to back, so a pass over a thread's vertices costs a few memory latencies
// rather than one per vertex.
__device__ __forceinline__ unsigned kw_ready(unsigned pend, const uint32_t (&wt)[32],
                                             const unsigned long long* word, unsigned p) {
  unsigned ready = 0, todo = pend;
  while (todo) {
    int as[8];
    unsigned long long wv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      as[k] = -1;
      if (todo) {
        as[k] = __ffs(todo) - 1;
        todo &= todo - 1;
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      wv[k] = 0;
      if (as[k] >= 0) {
        const uint32_t b = wt[as[k]];
        wv[k] = b == kNone ? ((unsigned long long)p << 48) : ld_relaxed(&word[b]);
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (as[k] >= 0 && tag_of(wv[k]) == p) ready |= 1u << as[k];
  }
  return ready;
}

}  // namespace
}  // namespace sco
