// batch.cu -- the per-step path of Fig. 1 for a batch of replicas: every phase is one
// launch over all replicas, and every size that depends on the switched graph (CSR
// entries, Delta, KW levels, colour count) is read on the device, so a run of steps needs
// no host round trip and can be captured in one CUDA graph.
//
// Per step: (A) switch + CSR of every replica (Sec. 2.1), (2) Kuhn-Wattenhofer colouring of
// every replica's graph (Sec. 2.3.3) and global colour classes (sites of all replicas sorted
// by (colour, global index)), (3) one persistent cooperative kernel that walks the colours
// in ascending order; class c of the batch is the union of every replica's class c, and a
// grid barrier separates colours.  Each site takes exactly the decisions of a single-lattice
// run (same per-site code, same random streams), so replica r is bit-identical to a
// single-lattice run with its parameters.
//
// Buffers that can overflow (CSR entries, overflow half-edges, palette) are checked on the
// device; a step that would overflow sets a replan flag before touching the spins, every
// later kernel returns at once, and the host grows the buffers and repeats that step.
#include <cstdint>

#include "batch.h"
#include "grid_dev.cuh"
#include "kw_bcr.cuh"
#include "kw_dev.cuh"
#include "sweep_dev.cuh"
#include "switch_dev.cuh"

namespace sco {

namespace {

__device__ __forceinline__ bool halted(const BatchDev& B) {
  return ld_status(&B.ctl->flag) != 0 || ld_status(&B.ctl->status) != 0;
}

// Block-uniform halt test (thread 0 reads, the block agrees).
__device__ __forceinline__ bool block_halted(const BatchDev& B) {
  __shared__ int h;
  if (threadIdx.x == 0) h = halted(B) ? 1 : 0;
  __syncthreads();
  return h != 0;
}

// Replica of this block in the per-site launches (kBatchBlock sites per block).
__device__ __forceinline__ int block_replica(const BatchDev& B) {
  return find_le(B.blk_start, B.R, blockIdx.x);
}

// ---- step (A): switch + CSR -------------------------------------------------------------

__global__ void __launch_bounds__(256) kb_clear(const BatchDev B) {
  if (block_halted(B)) return;
  for (int r = threadIdx.x; r < B.R; r += blockDim.x) {
    DevCounters& c = B.cnt[r];
    c.n_half = 0;
    c.n_dip = 0;
    c.ovf_n = 0;
    c.nnz = 0;
    c.max_degree = 0;
    c.max_degree_dip = 0;
    c.n_colours = 0;
    for (int p = 0; p < 32; ++p) c.lev_rounds[p] = 0;
  }
  if (threadIdx.x == 0) {
    B.ctl->ovf_n = 0;
    B.ctl->ovf_full = 0;
  }
}

template <int PREC>
__global__ void __launch_bounds__(256, 4) kb_switch(const BatchDev B) {
  if (block_halted(B)) return;
  __shared__ uint64_t sW[kNear];
  __shared__ uint32_t sD[kNear];
  __shared__ DevParams sP;
  const int r = block_replica(B);
  const RepDesc* d = B.desc + r;
  smem_copy(&sP, &d->P, sizeof(DevParams));
  __syncthreads();
  const int64_t K = sP.K;
  const int64_t nnear = K < kNear ? K : kNear;
  const uint64_t* W = d->W;
  const uint32_t* disp = d->disp;
  for (int q = threadIdx.x; q < nnear; q += blockDim.x) {
    sW[q] = W[q];
    sD[q] = disp[q];
  }
  __syncthreads();
  const NearTable T{sW, sD, W, disp, nnear, K, nnear};
  const uint32_t base = d->base;
  const uint32_t i = (blockIdx.x - B.blk_start[r]) * kBatchBlock + threadIdx.x;
  unsigned long long n_half = 0, n_dip = 0;
  unsigned ghits = 0, g32 = 0;
  if (i < (uint32_t)sP.N) {
    const uint32_t gs = base + i;
    const uint64_t Wtot = K > 0 ? __ldg(&W[K - 1]) : 0;
    const uint32_t epoch = (uint32_t)(B.ctl->step / (unsigned long long)B.n_sw);
    const SwitchOut o{B.hslot, B.indeg + base, B.ovf, B.ovf_cap, &B.ctl->ovf_n,
                      &B.ctl->ovf_full};
    const size_t so = 3 * (size_t)base;
    const uint32_t n_out =
        switch_site<PREC>(sP, T, Wtot, d->sw64, d->xyq, d->xy32, B.s + so, B.s32 + base, epoch,
                          d->mnn0, d->mnn1, i, gs, o, n_dip, ghits, g32);
    B.hcnt[gs] = n_out;
    n_half = n_out;
  }
  n_half = warp_sum_u64(n_half);
  n_dip = warp_sum_u64(n_dip);
  const unsigned long long gh = warp_sum_u64(ghits), gl = warp_sum_u64(g32);
  if ((threadIdx.x & 31) == 0) {
    DevCounters* c = B.cnt + r;
    if (n_half) atomicAdd(&c->n_half, n_half);
    if (n_dip) atomicAdd(&c->n_dip, n_dip);
    if (gh) atomicAdd(&c->guard_fp64, gh);
    if (gl) atomicAdd(&c->guard_fp32, gl);
  }
}

__global__ void __launch_bounds__(256) kb_degree(const BatchDev B) {
  if (block_halted(B)) return;
  const int r = block_replica(B);
  const uint32_t base = B.site_start[r], N = B.site_start[r + 1] - base;
  const uint32_t i = (blockIdx.x - B.blk_start[r]) * kBatchBlock + threadIdx.x;
  unsigned m = 0;
  if (i < N) {
    const uint32_t gs = base + i;
    m = B.hcnt[gs] + B.indeg[gs];
    B.deg[gs] = m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(&B.cnt[r].max_degree, m);
}

// Per-replica palette and KW levels; capacity checks (sets the replan flag).
__global__ void __launch_bounds__(1024) kb_plan(const BatchDev B) {
  if (block_halted(B)) return;
  __shared__ unsigned sg, sl;
  if (threadIdx.x == 0) {
    sg = 0;
    sl = 0;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < B.R; r += blockDim.x) {
    const uint32_t base = B.site_start[r], N = B.site_start[r + 1] - base;
    const uint32_t g = B.cnt[r].max_degree + 1;
    const unsigned long long G = ((unsigned long long)N + g - 1) / g;
    unsigned M = 0;
    while ((1ull << M) < G) ++M;
    B.plan[r] = RepPlan{g, M, div_magic(g)};
    B.cnt[r].g = g;
    B.cnt[r].levels = M;
    B.cnt[r].nnz = (unsigned long long)(B.row_ptr[base + N] - B.row_ptr[base]);
    atomicMax(&sg, g);
    atomicMax(&sl, M);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    BatchCtl* c = B.ctl;
    c->gmax = sg;
    c->lmax = sl;
    int f = 0;
    if (c->nnz > B.col_cap) {
      f |= kReplanCol;
      c->need_col = c->nnz;
    }
    if (c->ovf_full) f |= kReplanOvf;
    if (sg > B.pal_cap) f |= kReplanPal;
    if (f) atomicOr(&c->flag, f);
  }
}

__global__ void __launch_bounds__(256) kb_fill(const BatchDev B) {
  if (block_halted(B)) return;
  const int r = block_replica(B);
  const uint32_t base = B.site_start[r], N = B.site_start[r + 1] - base;
  const uint32_t i = (blockIdx.x - B.blk_start[r]) * kBatchBlock + threadIdx.x;
  if (i >= N) return;
  const uint32_t gs = base + i;
  const uint32_t n = min(B.hcnt[gs], (uint32_t)kSlotCap);
  const uint32_t up = B.row_ptr[gs] + B.indeg[gs];
  for (uint32_t q = 0; q < n; ++q) {
    const uint32_t jv = B.hslot[(size_t)gs * kSlotCap + q];
    const uint32_t jg = base + (jv & kIndexMask);
    B.col[up + q] = jv;
    B.col[B.row_ptr[jg] + atomicAdd(&B.lcur[jg], 1u)] = i | (jv & kExchOnly);
  }
}

__global__ void __launch_bounds__(256) kb_fill_ovf(const BatchDev B) {
  if (block_halted(B)) return;
  unsigned long long n = B.ctl->ovf_n;
  if (n > B.ovf_cap) n = B.ovf_cap;
  for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n;
       q += (unsigned long long)gridDim.x * blockDim.x) {
    const uint32_t gs = B.ovf[2 * q], jv = B.ovf[2 * q + 1];
    const int r = find_le(B.site_start, B.R, gs);
    const uint32_t base = B.site_start[r];
    const uint32_t jg = base + (jv & kIndexMask);
    B.col[B.row_ptr[gs] + B.indeg[gs] + kSlotCap + atomicAdd(&B.ocur[gs], 1u)] = jv;
    B.col[B.row_ptr[jg] + atomicAdd(&B.lcur[jg], 1u)] = (gs - base) | (jv & kExchOnly);
  }
}

__global__ void __launch_bounds__(256) kb_rowsort(const BatchDev B) {
  if (block_halted(B)) return;
  const int r = block_replica(B);
  const uint32_t base = B.site_start[r], N = B.site_start[r + 1] - base;
  const uint32_t i = (blockIdx.x - B.blk_start[r]) * kBatchBlock + threadIdx.x;
  unsigned nd = 0;
  if (i < N) {
    const uint32_t gs = base + i;
    nd = sort_row(B.col + B.row_ptr[gs], B.row_ptr[gs + 1] - B.row_ptr[gs]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nd = max(nd, __shfl_down_sync(0xffffffffu, nd, o));
  if ((threadIdx.x & 31) == 0 && nd) atomicMax(&B.cnt[r].max_degree_dip, nd);
}

// ---- step (2): colouring and classes ----------------------------------------------------

__global__ void __launch_bounds__(256) kb_kw_init(const BatchDev B) {
  if (block_halted(B)) return;
  const int r = block_replica(B);
  const uint32_t base = B.site_start[r], N = B.site_start[r + 1] - base;
  const uint32_t i = (blockIdx.x - B.blk_start[r]) * kBatchBlock + threadIdx.x;
  if (i >= N) return;
  const RepPlan pl = B.plan[r];
  const uint32_t c = i - fdiv(i, pl.magic) * pl.g;
  B.word[base + i] = pack(0, 0, c);
  B.col8[base + i] = (uint8_t)c;
  B.blk[base + i] = kNone;
}

// One KW level for every replica.  The right-half slots of all replicas at level p are
// numbered consecutively (a block-local scan of the per-replica counts); thread t owns
// slots t + k * nthreads and recolours their vertices as in the single-lattice kernel.
__global__ void __launch_bounds__(256, 4) kb_kw_level(const BatchDev B, unsigned p,
                                                    uint32_t low_gmax) {
  if (block_halted(B)) return;
  extern __shared__ uint32_t ksm[];
  const int R = B.R;
  uint32_t* rp = ksm;               // R + 1 slot prefix at level p
  uint32_t* sbase = rp + R + 1;     // R + 1 site bases
  uint32_t* smax = sbase + R + 1;   // R deepest round reached in this block
  const unsigned long long t_start = global_ns();
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    const RepPlan pl = B.plan[r];
    const uint32_t b0 = B.site_start[r], N = B.site_start[r + 1] - b0;
    uint32_t n = 0;
    if (p <= pl.levels && p > kw_low_levels(pl.g, pl.levels, low_gmax)) {
      const unsigned long long gsz = (unsigned long long)pl.g << p;
      n = (uint32_t)(((unsigned long long)N + gsz - 1) / gsz * ((unsigned long long)pl.g << (p - 1)));
    }
    rp[r] = n;
    sbase[r] = b0;
    smax[r] = 0;
  }
  if (threadIdx.x == 0) sbase[R] = B.site_start[R];
  __syncthreads();
  block_scan_excl(rp, R);
  const uint32_t Rtot = rp[R];
  const uint32_t nth = gridDim.x * blockDim.x;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t m = Rtot > tid ? (Rtot - tid + nth - 1) / nth : 0;  // owned slots
  auto vertex_of = [&](uint32_t slot) -> uint32_t {  // global vertex of a slot, kNone if >= N
    const int r = find_le(rp, R, slot);
    const RepPlan pl = B.plan[r];
    const uint32_t v = kw_vertex(slot - rp[r], pl.g << (p - 1), p, pl.magic);
    return v < sbase[r + 1] - sbase[r] ? sbase[r] + v : kNone;
  };
  // one attempt on global vertex gv; kNone once recoloured
  auto attempt = [&](uint32_t gv, bool& done) -> bool {
    const int r = find_le(sbase, R, gv);
    const uint32_t base = sbase[r], v = gv - base;
    unsigned long long* word = B.word + base;
    uint32_t* blk = B.blk + base;
    done = false;
    const uint32_t b = blk[v];
    if (b != kNone && tag_of(ld_relaxed(&word[b])) != p) return false;  // blocker unfinished
    unsigned rm = 0;
    const uint32_t w = kw_attempt(v, (uint32_t)(word[v] & kColMask), p, B.plan[r].magic,
                                  B.row_ptr + base, B.col, word, rm);
    blk[v] = w;
    if (w == kNone) {
      atomicMax(&smax[r], rm);
      done = true;
      return true;
    }
    return false;
  };
  unsigned nap = 64;
  if (m <= 32) {
    // global vertex, colour before the level, and the global index of the neighbour it waits
    // for (kNone: none recorded), per owned slot
    uint32_t vtx[32], cv[32], wt[32];
    unsigned pend = 0;
#pragma unroll
    for (int a = 0; a < 32; ++a) {
      vtx[a] = kNone;
      wt[a] = kNone;
      cv[a] = 0;
      if ((uint32_t)a < m) {
        vtx[a] = vertex_of(tid + a * nth);
        if (vtx[a] != kNone) {
          cv[a] = (uint32_t)(B.word[vtx[a]] & kColMask);
          pend |= 1u << a;
        }
      }
    }
    for (unsigned long long pass = 0; pend; ++pass) {
      bool progress = false;
      unsigned ready = kw_ready(pend, wt, B.word, p);
      while (ready) {
        const int a = __ffs(ready) - 1;
        ready &= ready - 1;
        const uint32_t gv = vtx[a];
        const int r = find_le(sbase, R, gv);
        const uint32_t base = sbase[r];
        unsigned rm = 0;
        const uint32_t w = kw_attempt(gv - base, cv[a], p, B.plan[r].magic, B.row_ptr + base,
                                      B.col, B.word + base, rm);
        if (w == kNone) {
          atomicMax(&smax[r], rm);
          pend &= ~(1u << a);
          progress = true;
          wt[a] = kNone;
        } else {
          wt[a] = base + w;
        }
      }
      if (!pend) break;
      if (progress) {
        nap = 64;
      } else {
        __nanosleep(nap);
        nap = nap < 2048 ? 2 * nap : 2048;
      }
      if ((pass & wait_pass_mask(B.ns_limit)) == wait_pass_mask(B.ns_limit) &&
          (global_ns() - t_start > B.ns_limit || ld_status(&B.ctl->status) != 0)) {
        atomicCAS(&B.ctl->status, 0, kStatusTimeout);
        break;
      }
    }
  } else {
    bool pending = true;
    for (unsigned long long pass = 0; pending; ++pass) {
      pending = false;
      bool progress = false;
      for (uint32_t k = 0; k < m; ++k) {
        const uint32_t gv = vertex_of(tid + k * nth);
        if (gv == kNone) continue;
        if (tag_of(B.word[gv]) == p) continue;
        bool done;
        attempt(gv, done);
        if (done) progress = true;
        else pending = true;
      }
      if (!pending) break;
      if (progress) {
        nap = 64;
      } else {
        __nanosleep(nap);
        nap = nap < 2048 ? 2 * nap : 2048;
      }
      if ((pass & wait_pass_mask(B.ns_limit)) == wait_pass_mask(B.ns_limit) &&
          (global_ns() - t_start > B.ns_limit || ld_status(&B.ctl->status) != 0)) {
        atomicCAS(&B.ctl->status, 0, kStatusTimeout);
        break;
      }
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x)
    if (smax[r]) atomicMax(&B.cnt[r].lev_rounds[p & 31], smax[r]);
}

// Final colours, and the colours in use per replica (bit sets).
__global__ void __launch_bounds__(256) kb_kw_final(const BatchDev B) {
  if (block_halted(B)) return;
  extern __shared__ uint32_t ubits[];
  const uint32_t nw = B.pal_cap / 32;
  for (uint32_t w = threadIdx.x; w < nw; w += blockDim.x) ubits[w] = 0;
  __syncthreads();
  const int r = block_replica(B);
  const uint32_t base = B.site_start[r], N = B.site_start[r + 1] - base;
  const uint32_t i = (blockIdx.x - B.blk_start[r]) * kBatchBlock + threadIdx.x;
  if (i < N) {
    const uint32_t c = (uint32_t)(B.word[base + i] & kColMask);
    B.colour[base + i] = c;
    if (c < B.pal_cap) atomicOr(&ubits[c >> 5], 1u << (c & 31));
  }
  __syncthreads();
  for (uint32_t w = threadIdx.x; w < nw; w += blockDim.x)
    if (ubits[w]) atomicOr(&B.used[(size_t)r * nw + w], ubits[w]);
}

__global__ void __launch_bounds__(1024) kb_colour_stats(const BatchDev B) {
  if (block_halted(B)) return;
  const uint32_t nw = B.pal_cap / 32;
  for (int r = threadIdx.x; r < B.R; r += blockDim.x) {
    DevCounters& c = B.cnt[r];
    unsigned n = 0;
    for (uint32_t w = 0; w < nw; ++w) n += __popc(B.used[(size_t)r * nw + w]);
    const RepPlan pl = B.plan[r];
    unsigned t = 0;
    for (unsigned p = 1; p <= pl.levels; ++p) t += c.lev_rounds[p & 31];
    c.n_colours = n;
    // plain BCR (2) spends exactly g rounds per level on the same colouring
    c.kw_rounds = B.desc[r].variant == 1 ? pl.g * pl.levels : t;
  }
}

constexpr uint32_t kTile = (uint32_t)kClassTileSites;

__global__ void __launch_bounds__(256) kb_tile_hist(const BatchDev B) {
  if (block_halted(B)) return;
  extern __shared__ uint32_t h[];
  const uint32_t P = B.pal_cap;
  for (uint32_t c = threadIdx.x; c < P; c += blockDim.x) h[c] = 0;
  __syncthreads();
  const uint32_t v0 = blockIdx.x * kTile;
  const uint32_t v1 = min(B.Ntot, v0 + kTile);
  for (uint32_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
    const uint32_t c = B.colour[v];
    if (c < P) atomicAdd(&h[c], 1u);
  }
  __syncthreads();
  for (uint32_t c = threadIdx.x; c < P; c += blockDim.x)
    B.tile_cnt[(size_t)c * B.ntiles + blockIdx.x] = h[c];
  if (blockIdx.x == 0 && threadIdx.x == 0) B.tile_cnt[(size_t)P * B.ntiles] = 0;
}

// One warp per tile of kTile global sites: stable placement, so that perm lists the sites
// of every class by increasing global index (replica, then site).
__global__ void __launch_bounds__(32) kb_tile_scatter(const BatchDev B) {
  if (block_halted(B)) return;
  extern __shared__ uint32_t run[];
  const uint32_t P = B.pal_cap;
  const int lane = threadIdx.x;
  for (uint32_t c = lane; c < P; c += 32) run[c] = B.tile_cnt[(size_t)c * B.ntiles + blockIdx.x];
  __syncwarp();
  const uint32_t v0 = blockIdx.x * kTile;
  const uint32_t v1 = min(B.Ntot, v0 + kTile);
  for (uint32_t vb = v0; vb < v1; vb += 32) {
    const uint32_t v = vb + lane;
    const uint32_t c0 = v < v1 ? B.colour[v] : 0xFFFFFFFFu;
    const bool ok = c0 < P;
    const uint32_t c = ok ? c0 : 0xFFFFFFFFu;
    const unsigned mask = __match_any_sync(0xffffffffu, c);
    if (ok) B.perm[run[c] + __popc(mask & ((1u << lane) - 1u))] = v;
    __syncwarp();
    if (ok && lane == __ffs(mask) - 1) run[c] += __popc(mask);
    __syncwarp();
  }
  if (blockIdx.x == 0) {
    for (uint32_t c = lane; c < P; c += 32) B.off[c] = B.tile_cnt[(size_t)c * B.ntiles];
    if (lane == 0) B.off[P] = B.Ntot;
  }
}

// ---- step (3): the colour-class sweep, one persistent kernel per MC step ----------------

// Proposals of every site of every replica for this MC step (see take_proposal).
__global__ void __launch_bounds__(256) kb_propose(const BatchDev B) {
  if (block_halted(B)) return;
  const int r = block_replica(B);
  const RepDesc* d = B.desc + r;
  const uint32_t base = B.site_start[r], N = B.site_start[r + 1] - base;
  const uint32_t i = (blockIdx.x - B.blk_start[r]) * kBatchBlock + threadIdx.x;
  if (i >= N) return;
  SiteCtx c;
  c.i = i;
  const bool ok = propose(d->P, c, B.ctl->step);
  B.prop[base + i] = ok ? make_double4_32a(c.Sn[0], c.Sn[1], c.Sn[2], c.u)
                        : make_double4_32a(0.0, 0.0, 1.0, -1.0);
}

// Sites of class c (all replicas) one per thread; undecided ones go to the deferred list of
// the colour; after a grid barrier one warp per deferred site settles it (FP64, then
// double-double); a second barrier closes the colour.
template <int PREC>
__global__ void __launch_bounds__(128, PREC == 1 ? 6 : 5) kb_sweep(const BatchDev B) {
  if (block_halted(B)) return;
  extern __shared__ uint32_t wsm[];
  const int R = B.R;
  uint32_t* sbase = wsm;          // R + 1
  uint32_t* sg1 = sbase + R + 1;  // R deferred by the first screen
  uint32_t* sg2 = sg1 + R;        // R sent on to double-double (FP32-guarded form)
  for (int r = threadIdx.x; r <= R; r += blockDim.x) sbase[r] = B.site_start[r];
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    sg1[r] = 0;
    sg2[r] = 0;
  }
  __syncthreads();
  const uint32_t gmax = B.ctl->gmax;
  const uint32_t nth = gridDim.x * blockDim.x;
  const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const uint32_t gwarp = gtid >> 5, nwarps = nth >> 5;
  for (uint32_t c = 0; c < gmax; ++c) {
    const uint32_t b = B.off[c], e = B.off[c + 1];
    for (uint32_t idx = b + gtid; idx < e; idx += nth) {
      const uint32_t gs = B.perm[idx];
      const int r = find_le(sbase, R, gs);
      const uint32_t base = sbase[r];
      const RepDesc* d = B.desc + r;
      const DevParams& P = d->P;
      const size_t so = 3 * (size_t)base;
      double* s = B.s + so;
      float4* s32 = B.s32 + base;
      SiteCtx x;
      load_site(P, x, gs - base, s);
      if (!take_proposal(x, B.prop + base)) {
        B.acc[gs] = 0;
        continue;
      }
      int dec = 1;
      if (x.u != 0.0) {
        dec = PREC == 1 ? accept_fp32(P, x, d->sw32, s32, B.row_ptr + base, B.col)
                        : accept_fp64(P, x, d->sw64, s, B.row_ptr + base, B.col);
      }
      if (dec == 2) {
        B.defer[b + atomicAdd(&B.dcnt[c], 1u)] = gs;
        atomicAdd(&sg1[r], 1u);
        continue;
      }
      write_site(P, x, dec == 1, s, PREC == 1 ? s32 : nullptr, B.acc + base);
    }
    if (!grid_sync(B.ctl->bar, &B.ctl->status, B.ns_limit)) break;
    const uint32_t nd = ld_u32_gpu(&B.dcnt[c]);
    if (nd == 0) continue;
    for (uint32_t q = gwarp; q < nd; q += nwarps) {
      const uint32_t gs = ld_u32_gpu(&B.defer[b + q]);
      const int r = find_le(sbase, R, gs);
      const uint32_t base = sbase[r];
      const RepDesc* d = B.desc + r;
      const DevParams& P = d->P;
      const size_t so = 3 * (size_t)base;
      double* s = B.s + so;
      float4* s32 = B.s32 + base;
      SiteCtx x;
      load_site(P, x, gs - base, s);
      take_proposal(x, B.prop + base);
      int dec = PREC == 1 ? accept_fp64_warp(P, x, d->sw64, s, B.row_ptr + base, B.col, lane) : 2;
      if (dec == 2) {
        if (PREC == 1 && lane == 0) atomicAdd(&sg2[r], 1u);
        dec = accept_dd_warp(P, x, s, B.row_ptr + base, B.col, lane) ? 1 : 0;
      }
      if (lane == 0) write_site(P, x, dec == 1, s, PREC == 1 ? s32 : nullptr, B.acc + base);
      __syncwarp();
    }
    if (!grid_sync(B.ctl->bar, &B.ctl->status, B.ns_limit)) break;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    DevCounters* cr = B.cnt + r;
    if (PREC == 1) {
      if (sg1[r]) atomicAdd(&cr->guard_fp32, (unsigned long long)sg1[r]);
      if (sg2[r]) atomicAdd(&cr->guard_fp64, (unsigned long long)sg2[r]);
    } else if (sg1[r]) {
      atomicAdd(&cr->guard_fp64, (unsigned long long)sg1[r]);
    }
  }
}

__global__ void kb_step_end(const BatchDev B) {
  if (threadIdx.x == 0 && !halted(B)) B.ctl->step += 1;
}

template <typename... Args>
cudaError_t launch_coop(void (*k)(Args...), unsigned grid, unsigned block, size_t smem,
                        cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

size_t kw_smem(int R) { return (size_t)(3 * R + 2) * sizeof(uint32_t); }

}  // namespace

size_t batch_sweep_smem(int R) { return (size_t)(3 * R + 1) * sizeof(uint32_t); }

int batch_kw_occupancy(int schedule, int R, unsigned pal) {
  int n = 0;
  const cudaError_t e =
      schedule == 0 && pal <= kBcrMaxPalette
          ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_kw_bcr<false>, 256, kw_bcr_smem(R, pal))
          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kb_kw_level, 256, kw_smem(R));
  if (e != cudaSuccess || n < 1) n = 1;
  return n;
}

cudaError_t batch_low_setup(int R, uint32_t gcap, int* blocks_per_sm, uint32_t* ecap) {
  int dev = 0, smem_sm = 0, smem_blk = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_kw_low, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_blk - 64);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_kw_low, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  if (kw_low_smem(R, gcap, 0) > (size_t)(smem_blk - 64)) return cudaErrorInvalidValue;
  int blocks = 1;
  kw_low_shape(R, gcap, (size_t)smem_sm, (size_t)(smem_blk - 64), &blocks, ecap);
  int occ = 0;  // what is resident in fact
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_kw_low, kLowThreads,
                                                    kw_low_smem(R, gcap, *ecap));
  if (e != cudaSuccess) return e;
  *blocks_per_sm = occ < 1 ? 1 : (occ < blocks ? occ : blocks);
  return cudaSuccess;
}

int batch_sweep_occupancy(int precision, int R) {
  int n = 0;
  cudaError_t e = precision == 1
                      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kb_sweep<1>, 128,
                                                                      batch_sweep_smem(R))
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kb_sweep<0>, 128,
                                                                      batch_sweep_smem(R));
  if (e != cudaSuccess || n < 1) n = 1;
  return n;
}

cudaError_t batch_switch(const BatchDev& B, const BatchLaunch& L, cudaStream_t st) {
  cudaError_t e;
  kb_clear<<<1, 256, 0, st>>>(B);
  if ((e = cudaMemsetAsync(B.indeg, 0, (size_t)B.Ntot * sizeof(uint32_t), st)) != cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(B.lcur, 0, (size_t)B.Ntot * sizeof(uint32_t), st)) != cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(B.ocur, 0, (size_t)B.Ntot * sizeof(uint32_t), st)) != cudaSuccess)
    return e;
  if (B.precision == 1) kb_switch<1><<<B.nblocks, kBatchBlock, 0, st>>>(B);
  else kb_switch<0><<<B.nblocks, kBatchBlock, 0, st>>>(B);
  kb_degree<<<B.nblocks, kBatchBlock, 0, st>>>(B);
  *L.launches += 3;
  if ((e = scan_excl_u32(B.deg, B.row_ptr, (int64_t)B.Ntot + 1, L.scan_tmp,
                         reinterpret_cast<uint64_t*>(&B.ctl->nnz), st, L.launches)) != cudaSuccess)
    return e;
  kb_plan<<<1, 1024, 0, st>>>(B);
  kb_fill<<<B.nblocks, kBatchBlock, 0, st>>>(B);
  kb_fill_ovf<<<2 * num_sms(), 256, 0, st>>>(B);
  kb_rowsort<<<B.nblocks, kBatchBlock, 0, st>>>(B);
  *L.launches += 4;
  return cudaGetLastError();
}

cudaError_t batch_colour(const BatchDev& B, const BatchLaunch& L, cudaStream_t st) {
  cudaError_t e;
  const size_t nw = B.pal_cap / 32;
  if ((e = cudaMemsetAsync(B.used, 0, (size_t)B.R * nw * sizeof(uint32_t), st)) != cudaSuccess)
    return e;
  kb_kw_init<<<B.nblocks, kBatchBlock, 0, st>>>(B);
  ++*L.launches;
  const uint32_t low_gmax = L.kw_low != 0 ? L.low_gmax : 0u;
  if (low_gmax) {
    KwLowView W{};
    W.R = B.R;
    W.site_start = B.site_start;
    W.plan = B.plan;
    W.row_ptr = B.row_ptr;
    W.col = B.col;
    W.word = B.word;
    W.col8 = B.col8;
    W.cnt = B.cnt;
    W.halt = &B.ctl->flag;
    W.gmax = low_gmax;
    W.gcap = low_gmax;
    W.ecap = L.low_ecap;
    k_kw_low<<<(unsigned)L.low_grid, kLowThreads, kw_low_smem(B.R, low_gmax, L.low_ecap),
               st>>>(W);
    ++*L.launches;
  }
  if (L.kw_schedule == 0 && B.pal_cap <= kBcrMaxPalette && L.levels < kBcrMaxLevels) {
    if ((e = cudaMemsetAsync(B.bcnt, 0, (size_t)kBcrMaxLevels * B.pal_cap * sizeof(uint32_t),
                             st)) != cudaSuccess)
      return e;
    KwView V{};
    V.R = B.R;
    V.site_start = B.site_start;
    V.plan = B.plan;
    V.row_ptr = B.row_ptr;
    V.col = B.col;
    V.word = B.word;
    V.col8 = B.col8;
    V.list = B.blk;
    V.bcnt = B.bcnt;
    V.cnt = B.cnt;
    V.bar = B.ctl->bar;
    V.status = &B.ctl->status;
    V.halt = &B.ctl->flag;
    V.pal = B.pal_cap;
    V.levels = L.levels;
    V.ns_limit = B.ns_limit;
    V.imask = B.imask;
    V.imeta = B.imeta;
    V.ilist = B.ilist;
    V.gmax = &B.ctl->gmax;
    V.low_gmax = low_gmax;
    if ((e = launch_coop(k_kw_bcr<false>, (unsigned)L.kw_grid, 256, kw_bcr_smem(B.R, B.pal_cap), st,
                         V)) != cudaSuccess)
      return e;
    ++*L.launches;
  } else {
    for (unsigned p = 1; p <= L.levels; ++p) {
      if ((e = launch_coop(kb_kw_level, (unsigned)L.kw_grid, 256, kw_smem(B.R), st, B, p,
                           low_gmax)) != cudaSuccess)
        return e;
      ++*L.launches;
    }
  }
  kb_kw_final<<<B.nblocks, kBatchBlock, nw * sizeof(uint32_t), st>>>(B);
  kb_colour_stats<<<1, 1024, 0, st>>>(B);
  kb_tile_hist<<<B.ntiles, 256, (size_t)B.pal_cap * sizeof(uint32_t), st>>>(B);
  *L.launches += 3;
  if ((e = scan_excl_u32(B.tile_cnt, B.tile_cnt, (int64_t)B.pal_cap * B.ntiles + 1, L.scan_tmp,
                         nullptr, st, L.launches)) != cudaSuccess)
    return e;
  kb_tile_scatter<<<B.ntiles, 32, (size_t)B.pal_cap * sizeof(uint32_t), st>>>(B);
  ++*L.launches;
  return cudaGetLastError();
}

cudaError_t batch_sweep(const BatchDev& B, const BatchLaunch& L, cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(B.dcnt, 0, (size_t)B.pal_cap * sizeof(uint32_t), st)) != cudaSuccess)
    return e;
  kb_propose<<<B.nblocks, kBatchBlock, 0, st>>>(B);
  ++*L.launches;
  if (B.precision == 1)
    e = launch_coop(kb_sweep<1>, (unsigned)L.sweep_grid, 128, batch_sweep_smem(B.R), st, B);
  else
    e = launch_coop(kb_sweep<0>, (unsigned)L.sweep_grid, 128, batch_sweep_smem(B.R), st, B);
  ++*L.launches;
  return e;
}

cudaError_t batch_step_end(const BatchDev& B, const BatchLaunch& L, cudaStream_t st) {
  kb_step_end<<<1, 32, 0, st>>>(B);
  ++*L.launches;
  return cudaGetLastError();
}

}  // namespace sco
