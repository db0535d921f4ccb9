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
// cooperative kernel in which every thread recolours its own vertices once their larger
// neighbours are done: no grid-wide barrier between rounds,
// same colours as the synchronous rounds, and t_R recovered from the per-vertex rounds.
#include <algorithm>
#include <cstdint>

#include "kw_bcr.cuh"
#include "kw_dev.cuh"
#include "kw_low.cuh"

namespace sco {

namespace {

__global__ void k_kw_init(int64_t N, uint32_t g, unsigned long long* __restrict__ word,
                          uint8_t* __restrict__ col8, uint32_t* __restrict__ blk) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v < N) {
    const unsigned c = (unsigned)(v % g);
    word[v] = pack(0, 0, c);
    col8[v] = (uint8_t)c;
    blk[v] = 0xFFFFFFFFu;
  }
}

__global__ void __launch_bounds__(256, 4) k_kw_level(uint32_t N, uint32_t g, unsigned long long M,
                                                  unsigned p, const uint32_t* __restrict__ row_ptr,
                                                  const uint32_t* __restrict__ col,
                                                  unsigned long long* word,
                                                  uint32_t* __restrict__ blk,
                                                  DevCounters* __restrict__ cnt,
                                                  unsigned long long ns_limit) {
  const unsigned long long t_start = global_ns();
  const uint32_t half = g << (p - 1);
  const uint32_t ngroups = (uint32_t)(((unsigned long long)N + ((unsigned long long)g << p) - 1) /
                                      ((unsigned long long)g << p));
  const uint32_t R = ngroups * half;  // right-half slots (some beyond N)
  const uint32_t nth = gridDim.x * blockDim.x;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t m = R > tid ? (R - tid + nth - 1) / nth : 0;  // owned slots
  unsigned rmax = 0;
  unsigned nap = 64;  // back-off (ns) while nothing of this thread can progress
  if (m <= 32) {
    // one bit per unfinished owned vertex; the vertex, its colour before the level and the
    // neighbour it waits for (kNone: none recorded) stay with the thread
    uint32_t vtx[32], cv[32], wt[32];
    unsigned pend = 0;
#pragma unroll
    for (int a = 0; a < 32; ++a) {
      vtx[a] = kNone;
      wt[a] = kNone;
      cv[a] = 0;
      if ((uint32_t)a < m) {
        const uint32_t v = kw_vertex(tid + a * nth, half, p, M);
        if (v < N) {
          vtx[a] = v;
          cv[a] = (uint32_t)(word[v] & kColMask);
          pend |= 1u << a;
        }
      }
    }
    for (unsigned long long pass = 0; pend; ++pass) {
      bool progress = false;
      unsigned ready = kw_ready(pend, wt, word, p);
      while (ready) {
        const int a = __ffs(ready) - 1;
        ready &= ready - 1;
        const uint32_t w = kw_attempt(vtx[a], cv[a], p, M, row_ptr, col, word, rmax);
        wt[a] = w;
        if (w == kNone) {
          pend &= ~(1u << a);
          progress = true;
        }
      }
      if (!pend) break;
      if (progress) {
        nap = 64;
      } else {
        __nanosleep(nap);
        nap = nap < 2048 ? 2 * nap : 2048;
      }
      if ((pass & wait_pass_mask(ns_limit)) == wait_pass_mask(ns_limit) &&
          (global_ns() - t_start > ns_limit || ld_status(&cnt->status) != 0)) {
        // bounded wait: give up (SCO_ETIMEOUT) after ns_limit or once another thread failed
        atomicCAS(&cnt->status, 0, kStatusTimeout);
        break;
      }
    }
  } else {
    // many vertices per thread (very large lattices): every pass visits all owned slots
    bool pending = true;
    for (unsigned long long pass = 0; pending; ++pass) {
      pending = false;
      bool progress = false;
      for (uint32_t k = 0; k < m; ++k) {
        const uint32_t v = kw_vertex(tid + k * nth, half, p, M);
        if (v >= N) continue;
        const unsigned long long wv = word[v];
        if (tag_of(wv) == p) continue;
        const uint32_t b = blk[v];
        if (b != kNone && tag_of(ld_relaxed(&word[b])) != p) {
          pending = true;
          continue;
        }
        const uint32_t w = kw_attempt(v, (uint32_t)(wv & kColMask), p, M, row_ptr, col, word,
                                      rmax);
        blk[v] = w;
        if (w == kNone) progress = true;
        else pending = true;
      }
      if (!pending) break;
      if (progress) {
        nap = 64;
      } else {
        __nanosleep(nap);
        nap = nap < 2048 ? 2 * nap : 2048;
      }
      if ((pass & wait_pass_mask(ns_limit)) == wait_pass_mask(ns_limit) &&
          (global_ns() - t_start > ns_limit || ld_status(&cnt->status) != 0)) {
        atomicCAS(&cnt->status, 0, kStatusTimeout);
        break;
      }
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
  if (v < N) {
    // a completed colouring has every colour below g; after a wait that gave up (sticky
    // SCO_ETIMEOUT) an unfinished vertex may still hold one in [g, 2g): keep it inside the
    // palette so that the class construction and the sweeps stay in bounds
    const uint32_t c = (uint32_t)(word[v] & kColMask);
    colour[v] = c < g ? c : g - 1;
  }
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

// Colour classes: tiles of kClassTile sites count their (colour, degree bin) keys, an
// exclusive scan over (colour, tile, degree bin) gives every tile its start inside every class,
// and one warp per tile places its sites.  Inside a class the sites come tile by tile (so
// consecutive threads of a sweep visit nearby sites) and, inside a tile, by degree then index:
// the 32 lanes of a sweep warp then loop over rows of nearly equal length.  The order inside a
// class does not change any result (sites of one colour never interact).
constexpr int kClassTile = (int)kClassTileSites;

// degree bins per colour: a power of two with g * bins <= 8192 (32 KB of counters), at most 64
inline uint32_t deg_bins(uint32_t g) {
  uint32_t d = 64;
  while (d > 1 && (uint64_t)g * d > 8192) d >>= 1;
  return d;
}

__device__ __forceinline__ uint32_t class_key(uint32_t v, const uint32_t* __restrict__ colour,
                                              const uint32_t* __restrict__ row_ptr,
                                              uint32_t dk) {
  const uint32_t deg = row_ptr[v + 1] - row_ptr[v];
  return colour[v] * dk + min(deg, dk - 1);
}

__global__ void k_tile_hist(uint32_t N, uint32_t g, uint32_t dk, uint32_t ntiles,
                            const uint32_t* __restrict__ colour,
                            const uint32_t* __restrict__ row_ptr, uint32_t* __restrict__ tcnt) {
  extern __shared__ uint32_t h[];
  const uint32_t nk = g * dk;
  for (uint32_t k = threadIdx.x; k < nk; k += blockDim.x) h[k] = 0;
  __syncthreads();
  const uint32_t v0 = blockIdx.x * kClassTile;
  const uint32_t v1 = min(N, v0 + kClassTile);
  for (uint32_t v = v0 + threadIdx.x; v < v1; v += blockDim.x)
    atomicAdd(&h[class_key(v, colour, row_ptr, dk)], 1u);
  __syncthreads();
  for (uint32_t k = threadIdx.x; k < nk; k += blockDim.x) {
    const uint32_t c = k / dk, d = k - c * dk;
    tcnt[((size_t)c * ntiles + blockIdx.x) * dk + d] = h[k];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) tcnt[(size_t)nk * ntiles] = 0;
}

__global__ void __launch_bounds__(32) k_tile_scatter(uint32_t N, uint32_t g, uint32_t dk,
                                                     uint32_t ntiles,
                                                     const uint32_t* __restrict__ colour,
                                                     const uint32_t* __restrict__ row_ptr,
                                                     const uint32_t* __restrict__ base,
                                                     uint32_t* __restrict__ perm,
                                                     uint32_t* __restrict__ off) {
  extern __shared__ uint32_t run[];
  const int lane = threadIdx.x;
  const uint32_t nk = g * dk;
  for (uint32_t k = lane; k < nk; k += 32) {
    const uint32_t c = k / dk, d = k - c * dk;
    run[k] = base[((size_t)c * ntiles + blockIdx.x) * dk + d];
  }
  __syncwarp();
  const uint32_t v0 = blockIdx.x * kClassTile;
  const uint32_t v1 = min(N, v0 + kClassTile);
  for (uint32_t vb = v0; vb < v1; vb += 32) {
    const uint32_t v = vb + lane;
    const bool ok = v < v1;
    const uint32_t key = ok ? class_key(v, colour, row_ptr, dk) : 0xFFFFFFFFu;
    const unsigned mask = __match_any_sync(0xffffffffu, key);
    if (ok) perm[run[key] + __popc(mask & ((1u << lane) - 1u))] = v;
    __syncwarp();
    if (ok && lane == __ffs(mask) - 1) run[key] += __popc(mask);
    __syncwarp();
  }
  if (blockIdx.x == 0) {
    for (uint32_t c = lane; c < g; c += 32) off[c] = base[(size_t)c * ntiles * dk];
    if (lane == 0) off[g] = N;
  }
}

__global__ void k_nonempty_off(uint32_t g, const uint32_t* __restrict__ off,
                               DevCounters* __restrict__ cnt) {
  unsigned n = 0;
  for (uint32_t c = threadIdx.x; c < g; c += blockDim.x) n += off[c + 1] > off[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0 && n) atomicAdd(&cnt->n_colours, n);
}

// Fallback for palettes too large for shared memory: sites keep ascending order inside a
// warp and warps claim their ranges with atomics (the order inside a class does not affect
// the results: sites of one colour never interact).
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

// Parameters of the one-lattice view of the persistent colouring kernel.
__global__ void k_kw_meta(uint32_t N, uint32_t g, unsigned levels, unsigned long long magic,
                          uint32_t* site_start, RepPlan* plan) {
  site_start[0] = 0;
  site_start[1] = N;
  plan[0] = RepPlan{g, levels, magic};
}

// Blocks per SM and staged-edge capacity of the block-local level kernel for groups of gcap
// vertices (the first call lifts the kernel's shared-memory limit to the device maximum).
cudaError_t low_setup(uint32_t gcap, int* blocks_per_sm, uint32_t* ecap) {
  static int s_smem_sm = 0, s_smem_blk = 0;
  if (s_smem_sm == 0) {
    int dev = 0, a = 0, b = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&a, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&b, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_kw_low, cudaFuncAttributeMaxDynamicSharedMemorySize, b - 64);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_kw_low, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    s_smem_sm = a;
    s_smem_blk = b - 64;
  }
  int blocks = 1;
  kw_low_shape(1, gcap, (size_t)s_smem_sm, (size_t)s_smem_blk, &blocks, ecap);
  int occ = 0;  // what is resident in fact
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &occ, k_kw_low, kLowThreads, kw_low_smem(1, gcap, *ecap));
  if (e != cudaSuccess) return e;
  *blocks_per_sm = occ < 1 ? 1 : (occ < blocks ? occ : blocks);
  return cudaSuccess;
}

}  // namespace

// The split record build of a grid-wide level: k_kw_recw (warp-wide row reads; 6 blocks per SM
// at 39 registers) once a level-p group spans at least kRecWarpRows lattice rows, else k_kw_rec
// (a thread per vertex, 16 entries per chunk, 4 blocks per SM).  Per level at L = 2304 (g = 39)
// the thread kernel took 149, 192, 227, 255 ... 309 us for levels 7, 8, 9, 10 ... 17 (groups of
// 2.2, 4.3, 8.7, 17.3 ... rows), the warp kernel 237-249 us at every level.
constexpr int kRecChunk = 16, kRecBlocks = 4;
constexpr int kRecWBlocks = 6;
constexpr uint64_t kRecWarpRows = 12;

cudaError_t kw_run(const DevParams& P, const uint32_t* row_ptr, const uint32_t* col,
                   uint32_t g, int variant, ColourBufs& b, DevCounters* cnt,
                   unsigned long long ns_limit, cudaStream_t st, int64_t* launches) {
  const int64_t N = P.N;
  const int64_t G = (N + g - 1) / g;
  unsigned M = 0;  // levels (N < 2^30 keeps every index below 2^32)
  while (((int64_t)1 << M) < G) ++M;
  cudaError_t e = cudaMemsetAsync(cnt->lev_rounds, 0, sizeof(cnt->lev_rounds), st);
  if (e != cudaSuccess) return e;
  const unsigned nb = (unsigned)((N + 255) / 256);
  k_kw_init<<<nb, 256, 0, st>>>(N, g, b.word, b.col8, b.blk);
  ++*launches;
  unsigned long long magic = div_magic(g);
  uint32_t* site_start = reinterpret_cast<uint32_t*>(b.meta);
  RepPlan* plan = reinterpret_cast<RepPlan*>(b.meta + 2);
  k_kw_meta<<<1, 1, 0, st>>>((uint32_t)N, g, M, magic, site_start, plan);
  ++*launches;
  // levels 1..low: one block per group of g 2^low vertices
  const unsigned low = kw_low_levels(g, M, kLowMaxGroup);
  if (low > 0) {
    const uint32_t gcap = g << low;
    int lbps = 1;
    uint32_t ecap = 0;
    if ((e = low_setup(gcap, &lbps, &ecap)) != cudaSuccess) return e;
    const int64_t groups = (N + ((int64_t)g << low) - 1) / ((int64_t)g << low);
    const int64_t grid = std::min<int64_t>(groups, (int64_t)lbps * num_sms());
    KwLowView W{};
    W.R = 1;
    W.site_start = site_start;
    W.plan = plan;
    W.row_ptr = row_ptr;
    W.col = col;
    W.word = b.word;
    W.col8 = b.col8;
    W.cnt = cnt;
    W.halt = nullptr;
    W.gmax = kLowMaxGroup;
    W.gcap = gcap;
    W.ecap = ecap;
    k_kw_low<<<(unsigned)grid, kLowThreads, kw_low_smem(1, gcap, ecap), st>>>(W);
    ++*launches;
  }
  // Large lattices: all levels in one persistent kernel, buckets of equal previous colour in
  // turn (each thread would otherwise own many vertices per level).  Small ones: one kernel
  // per level in which a vertex recolours as soon as its larger neighbours are done (about g
  // grid barriers per level would dominate there).
  if (low >= M) {
    k_kw_final<<<nb, 256, 0, st>>>(N, M, g, variant, b.word, b.colour, cnt);
    ++*launches;
    return cudaGetLastError();
  }
  if (N >= (1 << 20) && g <= kBcrMaxPalette && M < kBcrMaxLevels) {
    const size_t sh = kw_bcr_smem(1, g);
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_kw_bcr<false>, 256, sh);
    if (e != cudaSuccess) return e;
    if (bps > 4) bps = 4;
    if (bps < 1) bps = 1;
    static int qbps = 0;  // the buckets-only instance
    if (qbps == 0) {
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&qbps, k_kw_bcr<true>, 256, sh)) !=
          cudaSuccess)
        return e;
      if (qbps > kBcrBucketBlocks) qbps = kBcrBucketBlocks;
      if (qbps < 1) qbps = 1;
    }
    if ((e = cudaMemsetAsync(b.bcnt, 0, (size_t)kBcrMaxLevels * g * sizeof(uint32_t), st)) !=
        cudaSuccess)
      return e;
    if ((e = cudaMemsetAsync(cnt->bar, 0, sizeof(cnt->bar), st)) != cudaSuccess) return e;
    KwView V{};
    V.R = 1;
    V.site_start = site_start;
    V.plan = plan;
    V.row_ptr = row_ptr;
    V.col = col;
    V.word = b.word;
    V.col8 = b.col8;
    V.list = b.blk;
    V.bcnt = b.bcnt;
    V.cnt = cnt;
    V.bar = cnt->bar;
    V.status = &cnt->status;
    V.halt = nullptr;
    V.pal = g;
    V.levels = M;
    V.ns_limit = ns_limit;
    V.imask = b.imask;
    V.imeta = b.imeta;
    V.ilist = b.ilist;
    V.gmax = nullptr;
    V.low_gmax = kLowMaxGroup;
    // buckets up to a quarter of the grid barrier-free, the larger ones one grid barrier apart
    // (all of them barrier-free measured 2.3 ms slower per step at L = 2304: the waiting
    // threads' polling slows the recolouring ones)
    V.free_max = 0;
    void* args[] = {(void*)&V};
    static int rbps = 0, tbps = 0;
    if (rbps == 0) {
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
               &rbps, k_kw_recw<kRecWBlocks>, 256, 0)) != cudaSuccess)
        return e;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
               &tbps, k_kw_rec<kRecChunk, kRecBlocks>, 256, 0)) != cudaSuccess)
        return e;
      if (rbps < 1) rbps = 1;
      if (tbps < 1) tbps = 1;
    }
    const int64_t wgrid = std::min<int64_t>((int64_t)rbps * num_sms(), kKwSplitBlocks);
    const int64_t tgrid = std::min<int64_t>((int64_t)tbps * num_sms(), kKwSplitBlocks);
    if (b.boff && g <= kLowMaxPal) {
      // per level: the records in two plain launches (k_kw_hist reserves, k_kw_recw builds),
      // then the cooperative kernel runs that level's buckets alone
      for (unsigned p = low + 1; p <= M; ++p) {
        // both launches of a level take the same grid (k_kw_hist's reservations are per block)
        const bool wide = ((uint64_t)g << p) >= kRecWarpRows * (uint64_t)P.Lx;
        const unsigned sgrid = (unsigned)(wide ? wgrid : tgrid);
        k_kw_hist<<<sgrid, 256, 0, st>>>(V, p, b.boff);
        if (wide)
          k_kw_recw<kRecWBlocks><<<sgrid, 256, 0, st>>>(V, p, b.boff);
        else
          k_kw_rec<kRecChunk, kRecBlocks><<<sgrid, 256, 0, st>>>(V, p, b.boff);
        V.p_only = p;
        V.prebuilt = 1;
        e = cudaLaunchCooperativeKernel((const void*)k_kw_bcr<true>,
                                        dim3((unsigned)(qbps * num_sms())), dim3(256), args, sh,
                                        st);
        if (e != cudaSuccess) return e;
        *launches += 3;
      }
    } else {
      e = cudaLaunchCooperativeKernel((const void*)k_kw_bcr<false>,
                                      dim3((unsigned)(bps * num_sms())), dim3(256), args, sh, st);
      if (e != cudaSuccess) return e;
      ++*launches;
    }
    k_kw_final<<<nb, 256, 0, st>>>(N, M, g, variant, b.word, b.colour, cnt);
    ++*launches;
    return cudaGetLastError();
  }
  static int blocks_per_sm = 0;
  if (blocks_per_sm == 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_kw_level, 256, 0);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  const int64_t want = (N / 2 + 255) / 256;
  int64_t grid = (int64_t)blocks_per_sm * num_sms();
  if (want < grid) grid = want > 0 ? want : 1;
  for (unsigned p = low + 1; p <= M; ++p) {
    uint32_t Nn = (uint32_t)N;
    uint32_t gg = g;
    unsigned pp = p;
    unsigned long long lim = ns_limit;
    void* args[] = {(void*)&Nn, (void*)&gg, (void*)&magic, (void*)&pp, (void*)&row_ptr,
                    (void*)&col, (void*)&b.word, (void*)&b.blk, (void*)&cnt, (void*)&lim};
    e = cudaLaunchCooperativeKernel((const void*)k_kw_level, dim3((unsigned)grid), dim3(256),
                                    args, 0, st);
    if (e != cudaSuccess) return e;
    ++*launches;
  }
  k_kw_final<<<nb, 256, 0, st>>>(N, M, g, variant, b.word, b.colour, cnt);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t bucket_run(const DevParams& P, uint32_t g, const uint32_t* row_ptr, ColourBufs& b,
                       DevCounters* cnt, cudaStream_t st, int64_t* launches) {
  const int64_t N = P.N;
  const uint32_t ntiles = (uint32_t)((N + kClassTile - 1) / kClassTile);
  if (g <= kMaxStablePalette) {
    cudaError_t e = cudaMemsetAsync(&cnt->n_colours, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const uint32_t dk = deg_bins(g);
    const size_t sh = (size_t)g * dk * sizeof(uint32_t);
    k_tile_hist<<<ntiles, 256, sh, st>>>((uint32_t)N, g, dk, ntiles, b.colour, row_ptr,
                                         b.tile_cnt);
    ++*launches;
    e = scan_excl_u32(b.tile_cnt, b.tile_cnt, (int64_t)g * dk * ntiles + 1, b.scan_tmp, nullptr,
                      st, launches);
    if (e != cudaSuccess) return e;
    k_tile_scatter<<<ntiles, 32, sh, st>>>((uint32_t)N, g, dk, ntiles, b.colour, row_ptr,
                                          b.tile_cnt, b.perm, b.off);
    ++*launches;
    k_nonempty_off<<<1, 1024, 0, st>>>(g, b.off, cnt);
    ++*launches;
    return cudaGetLastError();
  }
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
