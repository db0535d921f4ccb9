// kw_bcr.cuh -- all levels of the Kuhn-Wattenhofer colouring (Sec. 2.3.3) in one persistent
// cooperative kernel.  At each level the right-half vertices are bucketed by their colour
// from the previous level, and the buckets are processed from the largest colour down, one
// grid barrier apart: the order of plain colour reduction (2) of Sec. 2.3.2.
//
// When bucket c runs, every same-group right-half neighbour of larger previous colour has
// taken its new colour and the smaller ones still hold colours >= g (ignored), so each vertex
// of the bucket recolours at once to the smallest colour not held by a final same-group
// neighbour, with round 1 + the largest round among the larger ones.  That is the
// order-independent result of the modified reduction (2)': the same colouring and the same
// t_R as the synchronous rounds, for one lattice or a batch of them.
#pragma once

#include <cstdint>

#include "batch.h"
#include "grid_dev.cuh"
#include "kw_dev.cuh"
#include "kw_low.cuh"

namespace sco {
namespace {

constexpr unsigned kBcrMaxPalette = 2048;  // bucket counters kept in shared memory
constexpr unsigned kBcrMaxLevels = 32;

struct KwView {
  int R;                        // lattices (1 for a single lattice)
  const uint32_t* site_start;   // R + 1 first vertex of each lattice
  const RepPlan* plan;          // R: g, levels, magic
  const uint32_t* row_ptr;      // global entry offsets; col entries lattice-local
  const uint32_t* col;
  unsigned long long* word;     // packed (level, round, colour), global vertex index
  uint8_t* col8;                // colour (low byte) beside the words (null: words only)
  uint32_t* list;               // bucketed right-half vertices of the current level
  uint32_t* bcnt;               // kBcrMaxLevels x pal bucket sizes, zero on entry
  DevCounters* cnt;             // R: lev_rounds
  unsigned* bar;                // grid barrier words
  int* status;                  // sticky error word
  const int* halt;              // optional: nonzero on entry -> return at once
  unsigned pal;                 // >= every g, <= kBcrMaxPalette
  unsigned levels;              // >= every M, <= kBcrMaxLevels - 1
  unsigned long long ns_limit;  // bound of every barrier wait
  // Per-level records of the bucketed vertices (optional: null keeps the row path).  Item q
  // of the current level: the colours of its left-half same-group neighbours (imask, final
  // at this level), and its same-group right-half neighbours of larger previous colour
  // (ilist[kItemList q ..], global indices; imeta = their count, or kItemSlow above that).
  unsigned long long* imask;
  uint32_t* imeta;
  uint32_t* ilist;
  const unsigned* gmax;         // optional: largest palette on the device (else pal)
  uint32_t low_gmax;            // levels 1..kw_low_levels(g, M, low_gmax) done block-locally
  // buckets of at most this many vertices (record path) run without grid barriers between
  // them, each item waiting for its listed larger neighbours; 0: a quarter of the grid
  uint32_t free_max;
  // split record build (one lattice): run level p_only alone (0: every level), and with
  // prebuilt its buckets, list and records come from k_kw_hist and k_kw_recw
  unsigned p_only;
  int prebuilt;
};

constexpr int kItemList = kKwItemList;
// blocks per SM of the buckets-only instance (64 registers): with the overflow path out of line
// and lists read 8 entries at a time, 4 blocks measured best at L = 2304 (colour 7.23 ms per step
// against 7.42 for 3 blocks and 16 entries, 7.23 for 5 blocks)
constexpr int kBcrBucketBlocks = 4;
constexpr int kItemChunk = 8;  // listed neighbours loaded together
constexpr uint32_t kItemSlow = 0x100;

__device__ __forceinline__ uint4 ld_relaxed_v4(const uint32_t* p) {
  uint4 v;
  asm volatile("ld.relaxed.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}

// Builds the record of item pos (vertex gv, previous colour c) at level p, while every colour
// still holds its value from level p - 1: left-half same-group neighbours go into the mask
// (their colours are final at this level), right-half ones of larger previous colour into the
// list; smaller ones are ignored (they keep colours >= g while gv's bucket runs).  Palettes
// of at most 64 colours.  The row is read kChunk entries at a time.
template <int kChunk = 16>
__device__ __forceinline__ void kw_item_build(const KwView& V, uint32_t pos, uint32_t gv,
                                              uint32_t base, uint32_t c, unsigned p,
                                              const RepPlan& pl) {
  const uint32_t v = gv - base;
  // v's level-p group is [lo, lo + gsz), its left half [lo, lo + half)
  const uint32_t gsz = pl.g << p, half = pl.g << (p - 1);
  const uint32_t lo = (fdiv(v, pl.magic) >> p) * gsz;
  const uint32_t b = V.row_ptr[gv], e = V.row_ptr[gv + 1];
  const uint8_t* col8 = V.col8 + base;
  unsigned long long mask = 0;
  uint32_t n = 0;
  uint32_t* out = V.ilist + (size_t)pos * kItemList;
  for (uint32_t q0 = b; q0 < e; q0 += kChunk) {
    uint32_t uu[kChunk], cc[kChunk];
#pragma unroll
    for (int a = 0; a < kChunk; ++a) uu[a] = q0 + a < e ? (V.col[q0 + a] & kIndexMask) : kNone;
#pragma unroll
    for (int a = 0; a < kChunk; ++a) {  // offsets inside the group (>= gsz: another group)
      cc[a] = 0;
      uu[a] = uu[a] - lo;
      if (uu[a] < gsz) cc[a] = ld_relaxed_u8(&col8[lo + uu[a]]);
    }
#pragma unroll
    for (int a = 0; a < kChunk; ++a) {
      if (uu[a] >= gsz) continue;
      const uint32_t cu = cc[a];
      if (uu[a] < half) {
        mask |= 1ull << (cu & 63);
      } else if (cu > c) {
        if (n < (uint32_t)kItemList) out[n] = base + lo + uu[a];
        ++n;
      }
    }
  }
  V.imask[pos] = mask;
  V.imeta[pos] = n > (uint32_t)kItemList ? kItemSlow : n;
}

// An item whose record overflowed (more larger neighbours than it lists): recoloured from its
// row, in a function of its own so that the row's registers stay out of the bucket loop.
__device__ __noinline__ bool kw_item_slow(uint32_t gv, uint32_t base, uint32_t cb, unsigned p,
                                          uint32_t g, unsigned long long magic, const KwView V,
                                          unsigned& rm, unsigned long long t_start);

// An item's record head, loaded ahead of its bucket (the list is read when it runs).
struct KwItem {
  uint32_t gv;    // global vertex (kNone: no item)
  uint32_t meta;  // listed neighbours, or kItemSlow
  uint32_t pos;   // record index
  unsigned long long mask;
};

__device__ __forceinline__ void kw_item_fetch(KwItem& it, const KwView& V, uint32_t pos) {
  it.pos = pos;
  it.gv = ld_u32_gpu(&V.list[pos]);
  it.meta = ld_u32_gpu(&V.imeta[pos]);
  it.mask = ld_relaxed(&V.imask[pos]);
}

// Recolours an item from its record: the listed neighbours are final (bounded wait otherwise,
// which the bucket order rules out); new colour = smallest one free of mask and their
// colours, round = 1 + their largest round.  The list is read kItemChunk entries at a time,
// then their words together.
__device__ __forceinline__ bool kw_item_recolour(const KwItem& it, const KwView& V, unsigned p,
                                                 unsigned& rmax, unsigned long long t_start) {
  const uint32_t n = it.meta;
  const uint32_t* src = V.ilist + (size_t)it.pos * kItemList;
  unsigned long long mask = it.mask;
  unsigned rv = 0;
  for (uint32_t a0 = 0; a0 < n; a0 += kItemChunk) {
    uint32_t u[kItemChunk];
#pragma unroll
    for (int a = 0; a < kItemChunk; a += 4) {
      uint4 x = make_uint4(0, 0, 0, 0);
      if (a0 + a < n) x = ld_relaxed_v4(src + a0 + a);
      u[a] = x.x;
      u[a + 1] = x.y;
      u[a + 2] = x.z;
      u[a + 3] = x.w;
    }
    unsigned long long ww[kItemChunk];
#pragma unroll
    for (int a = 0; a < kItemChunk; ++a) ww[a] = a0 + a < n ? ld_relaxed(&V.word[u[a]]) : 0;
#pragma unroll
    for (int a = 0; a < kItemChunk; ++a) {
      if (a0 + a >= n) continue;
      unsigned long long wu = ww[a];
      unsigned spins = 0;
      while (tag_of(wu) != p) {
        __nanosleep(64);
        wu = ld_relaxed(&V.word[u[a]]);
        if ((++spins & wait_spin_mask(V.ns_limit)) == 0 &&
            (global_ns() - t_start > V.ns_limit || ld_status(V.status) != 0)) {
          atomicCAS(V.status, 0, kStatusTimeout);
          return false;
        }
      }
      mask |= 1ull << ((uint32_t)(wu & kColMask) & 63);
      rv = max(rv, rnd_of(wu));
    }
  }
  const unsigned cn = (unsigned)(__ffsll((long long)~mask) - 1);
  rmax = max(rmax, rv + 1);
  st_relaxed(&V.word[it.gv], pack(p, rv + 1, cn));
  st_relaxed_u8(&V.col8[it.gv], cn);
  return true;
}

// The row of a vertex with its first sixteen neighbour entries, loaded ahead of its turn.
struct KwRow {
  uint32_t gv;  // global vertex (kNone: no item)
  uint32_t b, e;
  uint32_t uu[16];
};

__device__ __forceinline__ void kw_fetch(KwRow& w, uint32_t gv, const uint32_t* __restrict__ row_ptr,
                                         const uint32_t* __restrict__ col) {
  w.gv = gv;
  if (gv == kNone) return;
  w.b = row_ptr[gv];
  w.e = row_ptr[gv + 1];
#pragma unroll
  for (int a = 0; a < 16; ++a) w.uu[a] = w.b + a < w.e ? (col[w.b + a] & kIndexMask) : kNone;
}

// Recolours v (lattice-local; its row fetched in w) of previous colour c: the smallest colour
// not held by a final same-group neighbour, round 1 + the largest round among the right-half
// ones.  A same-group right-half neighbour of larger previous colour that is not done yet
// (which the bucket order rules out) would be waited for, bounded (false on timeout or
// error).  Neighbour words are loaded sixteen at a time, back to back.
__device__ __forceinline__ bool kw_recolour(uint32_t v, uint32_t c, const KwRow& w, unsigned p,
                                            uint32_t g, unsigned long long M,
                                            const uint32_t* __restrict__ col,
                                            unsigned long long* word, uint8_t* col8,
                                            unsigned& rmax, int* status,
                                            unsigned long long t_start,
                                            unsigned long long ns_limit) {
  // v's level-p group is [lo, lo + gsz), its left half [lo, lo + half)
  const uint32_t gsz = g << p, half = g << (p - 1);
  const uint32_t lo = (fdiv(v, M) >> p) * gsz;
  const uint32_t b = w.b, e = w.e;
  unsigned long long used[4] = {0, 0, 0, 0};  // colours < 256 (mex <= degree)
  unsigned rv = 0;
  for (uint32_t q0 = b; q0 < e; q0 += 16) {
    uint32_t uu[16];
    unsigned long long ww[16];
    if (q0 == b) {
#pragma unroll
      for (int a = 0; a < 16; ++a) uu[a] = w.uu[a];
    } else {
#pragma unroll
      for (int a = 0; a < 16; ++a) uu[a] = q0 + a < e ? (col[q0 + a] & kIndexMask) : kNone;
    }
#pragma unroll
    for (int a = 0; a < 16; ++a) {  // offsets inside the group (>= gsz: another group)
      ww[a] = 0;
      uu[a] = uu[a] - lo;
      if (uu[a] < gsz) ww[a] = ld_relaxed(&word[lo + uu[a]]);
    }
#pragma unroll
    for (int a = 0; a < 16; ++a) {
      if (uu[a] >= gsz) continue;
      unsigned long long wu = ww[a];
      const bool right = uu[a] >= half;
      if (right && tag_of(wu) != p) {
        if ((uint32_t)(wu & kColMask) < c) continue;  // smaller: still >= g
        unsigned spins = 0;
        while (tag_of(wu) != p) {
          __nanosleep(64);
          wu = ld_relaxed(&word[lo + uu[a]]);
          if ((++spins & wait_spin_mask(ns_limit)) == 0 &&
              (global_ns() - t_start > ns_limit || ld_status(status) != 0)) {
            atomicCAS(status, 0, kStatusTimeout);
            return false;
          }
        }
      }
      const uint32_t cu = (uint32_t)(wu & kColMask);
      if (right) rv = max(rv, rnd_of(wu));
      if (cu < 256) used[cu >> 6] |= 1ull << (cu & 63);
    }
  }
  unsigned cn = 0;
  if (e - b < 256) {
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      if (~used[x]) {
        cn = 64 * x + __ffsll((long long)~used[x]) - 1;
        break;
      }
    }
  } else {
    cn = mex_slow(v, p, M, col, word, b, e);
  }
  rmax = max(rmax, rv + 1);
  st_relaxed(&word[v], pack(p, rv + 1, cn));
  if (col8) st_relaxed_u8(&col8[v], cn);
  return true;
}

inline size_t kw_bcr_smem(int R, unsigned pal) {
  return (size_t)(3 * R + 2 + 4 * pal + 1) * sizeof(uint32_t);
}

__device__ __noinline__ bool kw_item_slow(uint32_t gv, uint32_t base, uint32_t cb, unsigned p,
                                          uint32_t g, unsigned long long magic, const KwView V,
                                          unsigned& rm, unsigned long long t_start) {
  KwRow w;
  kw_fetch(w, gv, V.row_ptr, V.col);
  return kw_recolour(gv - base, cb, w, p, g, magic, V.col, V.word + base, V.col8 + base, rm,
                     V.status, t_start, V.ns_limit);
}

// kBuckets: an instance that only runs the buckets of levels whose records the split kernels
// built (V.prebuilt set), held to fewer registers for more resident threads per bucket.
template <bool kBuckets>
__global__ void __launch_bounds__(256, kBuckets ? kBcrBucketBlocks : 3) k_kw_bcr(const KwView V) {
  __shared__ int s_halt;
  if (threadIdx.x == 0) s_halt = V.halt ? ld_status(V.halt) : 0;
  __syncthreads();
  if (s_halt) return;
  extern __shared__ uint32_t sm[];
  const int R = V.R;
  const unsigned pal = V.pal;
  uint32_t* sbase = sm;             // R + 1
  uint32_t* rp = sbase + R + 1;     // R + 1 right-half slot prefix at this level
  uint32_t* smax = rp + R + 1;      // R deepest round in this block
  uint32_t* hist = smax + R;        // pal this block's vertices per previous colour
  uint32_t* offb = hist + pal;      // pal this block's offset inside each bucket
  uint32_t* lcur = offb + pal;      // pal
  uint32_t* start = lcur + pal;     // pal + 1 bucket starts
  __shared__ unsigned s_old[1];
  for (int r = threadIdx.x; r <= R; r += blockDim.x) sbase[r] = V.site_start[r];
  const uint32_t nth = gridDim.x * blockDim.x;
  const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
  // records (instead of rows) when every palette fits a 64-bit mask
  const bool fast =
      kBuckets || (V.imask != nullptr && V.col8 != nullptr && (V.gmax ? *V.gmax : pal) <= 64u);
  bool ok = true;
  for (unsigned p = 1; p <= V.levels && ok; ++p) {
    if (V.p_only != 0 && p != V.p_only) continue;
    // right-half slots of every lattice at level p
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      const RepPlan pl = V.plan[r];
      const uint32_t N = sbase[r + 1] - sbase[r];
      uint32_t n = 0;
      if (p <= pl.levels && p > kw_low_levels(pl.g, pl.levels, V.low_gmax)) {
        const unsigned long long gsz = (unsigned long long)pl.g << p;
        n = (uint32_t)(((unsigned long long)N + gsz - 1) / gsz *
                       ((unsigned long long)pl.g << (p - 1)));
      }
      rp[r] = n;
      smax[r] = 0;
    }
    for (unsigned c = threadIdx.x; c < pal; c += blockDim.x) {
      hist[c] = 0;
      lcur[c] = 0;
    }
    __syncthreads();
    block_scan_excl(rp, R);
    const uint32_t Rtot = rp[R];
    if (Rtot == 0) {  // no lattice has this level left (the same in every block)
      __syncthreads();
      continue;
    }
    auto vertex_of = [&](uint32_t slot) -> uint32_t {
      const int r = find_le(rp, R, slot);
      const RepPlan pl = V.plan[r];
      const uint32_t v = kw_vertex(slot - rp[r], pl.g << (p - 1), p, pl.magic);
      return v < sbase[r + 1] - sbase[r] ? sbase[r] + v : kNone;
    };
    uint32_t* bc = V.bcnt + (size_t)p * pal;
    if (kBuckets || V.prebuilt) {
      for (unsigned c = threadIdx.x; c < pal; c += blockDim.x) start[c] = ld_u32_gpu(&bc[c]);
      __syncthreads();
      block_scan_excl(start, (int)pal);
    } else {
    // bucket sizes: block histograms, then one reservation per (block, colour)
    for (uint32_t slot = gtid; slot < Rtot; slot += nth) {
      const uint32_t gv = vertex_of(slot);
      if (gv != kNone)
        atomicAdd(&hist[fast ? ld_relaxed_u8(&V.col8[gv])
                             : (uint32_t)(ld_relaxed(&V.word[gv]) & kColMask)],
                  1u);
    }
    __syncthreads();
    for (unsigned c = threadIdx.x; c < pal; c += blockDim.x)
      offb[c] = hist[c] ? atomicAdd(&bc[c], hist[c]) : 0u;
    if (!grid_sync(V.bar, V.status, V.ns_limit)) {
      ok = false;
      break;
    }
    for (unsigned c = threadIdx.x; c < pal; c += blockDim.x) start[c] = ld_u32_gpu(&bc[c]);
    __syncthreads();
    block_scan_excl(start, (int)pal);
    for (uint32_t slot = gtid; slot < Rtot; slot += nth) {
      const uint32_t gv = vertex_of(slot);
      if (gv == kNone) continue;
      const uint32_t c =
          fast ? ld_relaxed_u8(&V.col8[gv]) : (uint32_t)(ld_relaxed(&V.word[gv]) & kColMask);
      const uint32_t pos = start[c] + offb[c] + atomicAdd(&lcur[c], 1u);
      V.list[pos] = gv;
      if (fast) {
        const int r = find_le(sbase, R, gv);
        kw_item_build(V, pos, gv, sbase[r], c, p, V.plan[r]);
      }
    }
    if (!grid_sync(V.bar, V.status, V.ns_limit)) {
      ok = false;
      break;
    }
    }
    // buckets from the largest previous colour down, one grid barrier apart.  Between its
    // arrival at a barrier and its wait, each thread fetches the row of its first item of the
    // next non-empty bucket (nothing there depends on the bucket being finished).
    const unsigned long long t_start = global_ns();
    auto next_bucket = [&](int c) {  // largest non-empty bucket below c, -1 if none
      for (--c; c >= 0; --c)
        if (start[c + 1] > start[c]) return c;
      return -1;
    };
    int c = next_bucket((int)pal);
    if (fast) {
      // one item: record-driven, or from its row when the record overflowed
      auto recolour = [&](KwItem& it, int cb) -> bool {
        const int r = find_le(sbase, R, it.gv);
        unsigned rm = 0;
        bool mine;
        if (it.meta & kItemSlow) {  // more larger neighbours than the record holds
          mine = kw_item_slow(it.gv, sbase[r], (uint32_t)cb, p, V.plan[r].g, V.plan[r].magic, V,
                              rm, t_start);
        } else {
          mine = kw_item_recolour(it, V, p, rm, t_start);
        }
        atomicMax(&smax[r], rm);
        return mine;
      };
      // the largest colours' buckets hold at most one block's worth of vertices each: block 0
      // takes that run alone, one __syncthreads apart, and one grid barrier publishes it.  The
      // one-lattice bucket instance leaves them to the barrier-free run below instead (4 to 14 us
      // less per level at L = 2304: the run's waits follow only the actual neighbours, not every
      // larger bucket).
      int ct = (int)pal;
      if (!kBuckets)
        while (ct > 0 && start[ct] - start[ct - 1] <= blockDim.x) --ct;
      if (c >= ct) {  // a non-empty tail
        if (blockIdx.x == 0) {
          bool mine = true;
          for (int cb = c; cb >= ct; --cb) {
            const uint32_t b0 = start[cb], n = start[cb + 1] - b0;
            if (n == 0) continue;
            if (mine && threadIdx.x < n) {
              KwItem it;
              kw_item_fetch(it, V, b0 + threadIdx.x);
              mine = recolour(it, cb);
            }
            __syncthreads();
          }
        }
        // false for every block once an error was reported (status read after the barrier)
        ok = grid_sync(V.bar, V.status, V.ns_limit);
        c = next_bucket(ct);
      }
      // the buckets below that hold at most free_max vertices each run with no barrier
      // between them: every thread takes their items in descending colour order and waits
      // (bounded) for the listed neighbours, all of larger colour, hence taken up earlier by
      // their own threads (no cycle of waits); one grid barrier publishes the run
      if (ok && c >= 0) {
        int cm = c;
        const uint32_t fmax = V.free_max ? V.free_max : nth / 4;
        while (cm >= 0 && start[cm + 1] - start[cm] <= fmax) --cm;
        if (cm < c) {
          const uint32_t hi = start[c + 1], lo = start[cm + 1];
          bool mine = true;
          int cb = c;
          for (uint32_t q = gtid; q < hi - lo && mine; q += nth) {
            const uint32_t pos = hi - 1 - q;
            while (pos < start[cb]) --cb;
            KwItem it;
            kw_item_fetch(it, V, pos);
            mine = recolour(it, cb);
          }
          ok = grid_sync(V.bar, V.status, V.ns_limit);
          c = next_bucket(cm + 1);
        }
      }
      KwItem it;
      it.gv = kNone;
      if (c >= 0 && gtid < start[c + 1] - start[c]) kw_item_fetch(it, V, start[c] + gtid);
      while (c >= 0 && ok) {
        const uint32_t b0 = start[c], n = start[c + 1] - b0;
        bool mine = true;
        for (uint32_t q = gtid; q < n && mine; q += nth) {
          if (q != gtid) kw_item_fetch(it, V, b0 + q);
          mine = recolour(it, c);
        }
        grid_arrive(V.bar, s_old);
        const int cn = next_bucket(c);
        it.gv = kNone;
        if (cn >= 0 && gtid < start[cn + 1] - start[cn]) kw_item_fetch(it, V, start[cn] + gtid);
        ok = grid_wait(V.bar, s_old, V.status, V.ns_limit);
        c = cn;
      }
    } else {
      KwRow w;
      w.gv = kNone;
      if (c >= 0 && gtid < start[c + 1] - start[c])
        kw_fetch(w, ld_u32_gpu(&V.list[start[c] + gtid]), V.row_ptr, V.col);
      while (c >= 0 && ok) {
        const uint32_t b0 = start[c], n = start[c + 1] - b0;
        bool mine = true;
        for (uint32_t q = gtid; q < n && mine; q += nth) {
          if (q != gtid) kw_fetch(w, ld_u32_gpu(&V.list[b0 + q]), V.row_ptr, V.col);
          const uint32_t gv = w.gv;
          const int r = find_le(sbase, R, gv);
          const uint32_t base = sbase[r];
          unsigned rm = 0;
          mine = kw_recolour(gv - base, (uint32_t)c, w, p, V.plan[r].g, V.plan[r].magic, V.col,
                             V.word + base, nullptr, rm, V.status, t_start, V.ns_limit);
          atomicMax(&smax[r], rm);
        }
        grid_arrive(V.bar, s_old);
        const int cn = next_bucket(c);
        w.gv = kNone;
        if (cn >= 0 && gtid < start[cn + 1] - start[cn])
          kw_fetch(w, ld_u32_gpu(&V.list[start[cn] + gtid]), V.row_ptr, V.col);
        // false for every block once an error was reported (status read after the barrier)
        ok = grid_wait(V.bar, s_old, V.status, V.ns_limit);
        c = cn;
      }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < R; r += blockDim.x)
      if (smax[r]) atomicMax(&V.cnt[r].lev_rounds[p & 31], smax[r]);
  }
}

// Split record build of level p for one lattice (V.R == 1), ahead of a k_kw_bcr launch that
// runs only that level's buckets.  Both kernels deal the right-half slots to their threads in
// the same grid-stride order, so that the reservation each block of k_kw_hist makes per colour
// is where k_kw_recw puts that block's items; inside a (block, colour) range the order is free
// (a bucket's vertices share a colour, hence no edge).  A plain launch with more resident
// threads than the cooperative kernel keeps more records' load chains in flight.
__device__ __forceinline__ uint32_t kw_split_slots(const RepPlan& pl, uint32_t N, unsigned p) {
  const unsigned long long gsz = (unsigned long long)pl.g << p;
  return (uint32_t)(((unsigned long long)N + gsz - 1) / gsz * ((unsigned long long)pl.g << (p - 1)));
}

__global__ void __launch_bounds__(256) k_kw_hist(const KwView V, unsigned p,
                                                 uint32_t* __restrict__ boff) {
  __shared__ uint32_t hist[kLowMaxPal];
  const RepPlan pl = V.plan[0];
  const uint32_t N = V.site_start[1] - V.site_start[0];
  const unsigned pal = V.pal;
  for (unsigned c = threadIdx.x; c < pal; c += blockDim.x) hist[c] = 0;
  __syncthreads();
  const uint32_t Rtot = kw_split_slots(pl, N, p), nth = gridDim.x * blockDim.x;
  for (uint32_t slot = blockIdx.x * blockDim.x + threadIdx.x; slot < Rtot; slot += nth) {
    const uint32_t v = kw_vertex(slot, pl.g << (p - 1), p, pl.magic);
    if (v < N) atomicAdd(&hist[V.col8[v]], 1u);
  }
  __syncthreads();
  uint32_t* bc = V.bcnt + (size_t)p * pal;
  for (unsigned c = threadIdx.x; c < pal; c += blockDim.x)
    boff[(size_t)blockIdx.x * pal + c] = hist[c] ? atomicAdd(&bc[c], hist[c]) : 0u;
}

// The records of level p, one thread per right-half vertex walking its own row (kw_item_build,
// kChunk entries at a time).  Cheaper than k_kw_recw at the low grid-wide levels, where most of a
// row leaves the vertex's group and is skipped after one compare.
template <int kChunk, int kMinBlocks>
__global__ void __launch_bounds__(256, kMinBlocks) k_kw_rec(const KwView V, unsigned p,
                                                            const uint32_t* __restrict__ boff) {
  __shared__ uint32_t start[kLowMaxPal + 1];
  __shared__ uint32_t lcur[kLowMaxPal];
  const RepPlan pl = V.plan[0];
  const uint32_t N = V.site_start[1] - V.site_start[0];
  const unsigned pal = V.pal;
  const uint32_t* bc = V.bcnt + (size_t)p * pal;
  for (unsigned c = threadIdx.x; c < pal; c += blockDim.x) {
    start[c] = bc[c];
    lcur[c] = 0;
  }
  __syncthreads();
  block_scan_excl(start, (int)pal);
  for (unsigned c = threadIdx.x; c < pal; c += blockDim.x)
    start[c] += boff[(size_t)blockIdx.x * pal + c];
  __syncthreads();
  const uint32_t Rtot = kw_split_slots(pl, N, p), nth = gridDim.x * blockDim.x;
  for (uint32_t slot = blockIdx.x * blockDim.x + threadIdx.x; slot < Rtot; slot += nth) {
    const uint32_t v = kw_vertex(slot, pl.g << (p - 1), p, pl.magic);
    if (v >= N) continue;
    const uint32_t c = V.col8[v];
    const uint32_t pos = start[c] + atomicAdd(&lcur[c], 1u);
    V.list[pos] = v;
    kw_item_build<kChunk>(V, pos, v, 0u, c, p, pl);
  }
}

// The records of level p (kw_item_build's), with the rows read by whole warps: the warp's 32
// slots are consecutive vertices of one right half (or of two), so their rows are one contiguous
// run of col, which the lanes read 32 entries at a time, each entry by one lane (coalesced).  A lane finds its entry's vertex in the warp's row prefix (in shared
// memory), classifies the neighbour as kw_item_build does, and adds it to that vertex's record: a
// left-half colour by an atomic OR into the vertex's mask, a larger right-half one into the list
// at the vertex's count plus its rank among the vertex's list entries of the round.  Grid and
// slot order as in k_kw_hist (its reservations hold).
template <int kMinBlocks>
__global__ void __launch_bounds__(256, kMinBlocks) k_kw_recw(const KwView V, unsigned p,
                                                             const uint32_t* __restrict__ boff) {
  constexpr int kW = 8;           // warps per block
  constexpr int kRecRounds = 4;   // rounds of 32 row entries loaded together
  __shared__ uint32_t start[kLowMaxPal + 1];
  __shared__ uint32_t lcur[kLowMaxPal];
  __shared__ uint32_t w_pre[kW][33];
  __shared__ uint32_t w_rb[kW][32], w_lo[kW][32], w_c[kW][32], w_pos[kW][32], w_n[kW][32];
  __shared__ uint32_t w_m[kW][2][32];
  const RepPlan pl = V.plan[0];
  const uint32_t N = V.site_start[1] - V.site_start[0];
  const unsigned pal = V.pal;
  const uint32_t* bc = V.bcnt + (size_t)p * pal;
  for (unsigned c = threadIdx.x; c < pal; c += blockDim.x) {
    start[c] = bc[c];
    lcur[c] = 0;
  }
  __syncthreads();
  block_scan_excl(start, (int)pal);
  for (unsigned c = threadIdx.x; c < pal; c += blockDim.x)
    start[c] += boff[(size_t)blockIdx.x * pal + c];
  __syncthreads();
  const uint32_t gsz = pl.g << p, half = pl.g << (p - 1);
  const uint32_t Rtot = kw_split_slots(pl, N, p), nth = gridDim.x * blockDim.x;
  const int w = threadIdx.x >> 5;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;  // lanes below this one
  const uint32_t* __restrict__ col = V.col;
  const uint8_t* __restrict__ col8 = V.col8;
  uint32_t* pre = w_pre[w];
  for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < Rtot; base += nth) {
    const uint32_t slot = base + lane;
    uint32_t v = kNone, len = 0;
    if (slot < Rtot) {
      const uint32_t vv = kw_vertex(slot, half, p, pl.magic);
      if (vv < N) {
        v = vv;
        const uint32_t c = col8[v];
        const uint32_t pos = start[c] + atomicAdd(&lcur[c], 1u);
        V.list[pos] = v;
        const uint32_t rb = V.row_ptr[v];
        len = V.row_ptr[v + 1] - rb;
        w_rb[w][lane] = rb;
        w_lo[w][lane] = (fdiv(v, pl.magic) >> p) * gsz;
        w_c[w][lane] = c;
        w_pos[w][lane] = pos;
      }
    }
    w_n[w][lane] = 0;
    w_m[w][0][lane] = 0;
    w_m[w][1][lane] = 0;
    uint32_t incl = len;  // inclusive prefix of the row lengths over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (uint32_t)o) incl += t;
    }
    pre[lane + 1] = incl;
    if (lane == 0) pre[0] = 0;
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    __syncwarp();
    uint32_t k = 0;  // the vertex (lane) of this lane's entry, nondecreasing over the rounds
    for (uint32_t t0 = 0; t0 < total; t0 += 32 * kRecRounds) {
      // kRecRounds rounds at a time: their row entries, then their neighbours' colours, are
      // loaded together
      uint32_t kk[kRecRounds], uu[kRecRounds], cu[kRecRounds];
#pragma unroll
      for (int r = 0; r < kRecRounds; ++r) {
        const uint32_t t = t0 + 32 * r + lane;
        kk[r] = 0;
        uu[r] = kNone;
        if (t < total) {
          while (pre[k + 1] <= t) ++k;
          kk[r] = k;
          uu[r] = col[w_rb[w][k] + (t - pre[k])];
        }
      }
#pragma unroll
      for (int r = 0; r < kRecRounds; ++r) {
        cu[r] = 0;
        if (uu[r] != kNone) {
          uu[r] = (uu[r] & kIndexMask) - w_lo[w][kk[r]];
          if (uu[r] < gsz) cu[r] = col8[w_lo[w][kk[r]] + uu[r]];
        }
      }
#pragma unroll
      for (int r = 0; r < kRecRounds; ++r) {
        const uint32_t tr = t0 + 32 * r, t = tr + lane;
        if (tr >= total) break;  // uniform
        const bool act = t < total;
        const uint32_t kr = kk[r], u = uu[r];
        bool inl = false;
        uint32_t seg = 0;
        if (act) {
          if (u < gsz) {
            if (u < half) atomicOr(&w_m[w][cu[r] >> 5][kr], 1u << (cu[r] & 31));
            else if (cu[r] > w_c[w][kr]) inl = true;
          }
          seg = pre[kr] > tr ? pre[kr] - tr : 0;  // first lane of vertex kr in this round
        }
        const uint32_t lm = __ballot_sync(0xffffffffu, inl);
        const uint32_t mine = lm & ~((1u << seg) - 1u);  // list entries of lanes >= seg
        uint32_t n0 = 0;
        if (act) n0 = w_n[w][kr];
        if (inl) {
          const uint32_t n = n0 + __popc(mine & lt);
          if (n < (uint32_t)kItemList)
            V.ilist[(size_t)w_pos[w][kr] * kItemList + n] = w_lo[w][kr] + u;
        }
        __syncwarp();
        // the last lane of vertex kr in this round adds the round's list entries to its count
        if (act && (t + 1 == pre[kr + 1] || lane == 31))
          w_n[w][kr] = n0 + __popc(mine & (lt | (1u << lane)));
        __syncwarp();
      }
    }
    if (v != kNone) {
      const uint32_t pos = w_pos[w][lane], n = w_n[w][lane];
      V.imask[pos] = (unsigned long long)w_m[w][0][lane] | ((unsigned long long)w_m[w][1][lane] << 32);
      V.imeta[pos] = n > (uint32_t)kItemList ? kItemSlow : n;
    }
    __syncwarp();
  }
}

}  // namespace
}  // namespace sco
