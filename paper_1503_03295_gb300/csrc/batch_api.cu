// batch_api.cu -- the C ABI of batched replicas (include/sco.h): set-up, graph capture and
// replay of runs of MC steps, device-side replanning, autotuning of result-invariant launch
// choices, and per-replica getters.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "batch.h"
#include "sco.h"

using namespace sco;

struct sco_batch {
  std::vector<sco_params> p;
  int R = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int64_t launches = 0, graph_launches = 0;
  int32_t replans = 0;
  std::vector<DevParams> P;
  std::vector<Table> lists;  // sorted list + hazard prefix, one per lattice shape
  std::vector<Table> xy;     // temperature-dependent tables, one per replica
  std::vector<uint32_t> site_start, blk_start;
  std::vector<RepDesc> desc;
  BatchDev B{};
  BatchLaunch L{};
  size_t scan_tmp_n = 0;  // elements the scan buffer serves
  DevCounters* hcnt = nullptr;  // pinned, R
  BatchCtl* hctl = nullptr;     // pinned
  int64_t t = 0;
  bool have_graph = false;
  int sticky = 0;
  sco_batch_tuning tune{};
  int kw_occ = 1, sweep_occ = 1;
  int low_occ = 1;        // resident blocks per SM of the block-local level kernel
  uint32_t low_ecap = 0;  // its staged-edge capacity
  struct Graph {
    cudaGraphExec_t exec;
    int64_t launches;  // kernels in one replay
  };
  std::map<std::pair<int64_t, int>, Graph> graphs;
  bool capture_ok = true;
};

namespace {

sco_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return SCO_OK;
  if (e == cudaErrorMemoryAllocation) return SCO_ENOMEM;
  return SCO_ECUDA;
}

#define SCO_TRY(expr)                            \
  do {                                           \
    const cudaError_t e_ = (expr);               \
    if (e_ != cudaSuccess) return from_cuda(e_); \
  } while (0)

constexpr uint32_t kPalMax = 8192;  // tile histograms stay within 32 KB of shared memory

void drop_graphs(sco_batch* b) {
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second.exec);
  b->graphs.clear();
}

void free_all(sco_batch* b) {
  drop_graphs(b);
  BatchDev& B = b->B;
  cudaFree((void*)B.desc);
  cudaFree(B.plan);
  cudaFree(B.cnt);
  cudaFree(B.ctl);
  cudaFree((void*)B.blk_start);
  cudaFree((void*)B.site_start);
  cudaFree(B.s);
  cudaFree(B.s32);
  cudaFree(B.acc);
  cudaFree(B.hslot);
  cudaFree(B.hcnt);
  cudaFree(B.indeg);
  cudaFree(B.deg);
  cudaFree(B.lcur);
  cudaFree(B.ocur);
  cudaFree(B.ovf);
  cudaFree(B.row_ptr);
  cudaFree(B.col);
  cudaFree(B.word);
  cudaFree(B.col8);
  cudaFree(B.blk);
  cudaFree(B.colour);
  cudaFree(B.used);
  cudaFree(B.tile_cnt);
  cudaFree(B.perm);
  cudaFree(B.off);
  cudaFree(B.defer);
  cudaFree(B.prop);
  cudaFree(B.imask);
  cudaFree(B.imeta);
  cudaFree(B.ilist);
  cudaFree(B.dcnt);
  cudaFree(B.bcnt);
  cudaFree(b->L.scan_tmp);
  for (auto& t : b->xy) table_free_xy(t);
  for (auto& t : b->lists) table_free(t);
  if (b->hcnt) cudaFreeHost(b->hcnt);
  if (b->hctl) cudaFreeHost(b->hctl);
  if (b->own_stream && b->st) cudaStreamDestroy(b->st);
}

// Buffers whose size follows the palette capacity.
cudaError_t alloc_palette(sco_batch* b, uint32_t pal) {
  BatchDev& B = b->B;
  cudaFree(B.used);
  cudaFree(B.tile_cnt);
  cudaFree(B.off);
  cudaFree(B.dcnt);
  cudaFree(B.bcnt);
  B.used = B.tile_cnt = B.off = B.dcnt = B.bcnt = nullptr;
  B.pal_cap = pal;
  cudaError_t e = cudaMalloc(&B.used, (size_t)b->R * (pal / 32) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&B.tile_cnt, ((size_t)pal * B.ntiles + 1) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&B.off, (pal + 1) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&B.dcnt, pal * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&B.bcnt, (size_t)32 * pal * sizeof(uint32_t));
  const size_t need = std::max((size_t)B.Ntot + 1, (size_t)pal * B.ntiles + 1);
  if (e == cudaSuccess && need > b->scan_tmp_n) {
    cudaFree(b->L.scan_tmp);
    b->L.scan_tmp = nullptr;
    e = cudaMalloc(&b->L.scan_tmp, scan_tmp_bytes((int64_t)need));
    if (e == cudaSuccess) b->scan_tmp_n = need;
  }
  return e;
}

void set_grids(sco_batch* b) {
  const int sms = num_sms();
  b->L.kw_schedule = b->tune.kw_schedule;
  b->L.kw_low = b->tune.kw_low;
  b->L.low_gmax = (uint32_t)b->tune.kw_low_group;
  if (batch_low_setup(b->R, b->L.low_gmax, &b->low_occ, &b->low_ecap) != cudaSuccess) {
    b->L.kw_low = 0;  // no block-local levels at this size (the level kernels take them)
    b->low_occ = 1;
    b->low_ecap = 0;
  }
  b->L.low_grid = b->low_occ * sms;
  b->L.low_ecap = b->tune.kw_low == 2 ? 0u : b->low_ecap;
  b->kw_occ = batch_kw_occupancy(b->tune.kw_schedule, b->R, b->B.pal_cap);
  b->L.kw_grid = std::min(b->tune.kw_blocks_per_sm, b->kw_occ) * sms;
  b->L.sweep_grid = std::min(b->tune.sweep_blocks_per_sm, b->sweep_occ) * sms;
}

// Enqueues MC steps t0 .. t0 + k - 1 (switch + colour at epoch starts).
cudaError_t enqueue_steps(sco_batch* b, int64_t t0, int k) {
  cudaError_t e = cudaSuccess;
  const int n_sw = b->p[0].n_sw;
  for (int q = 0; q < k && e == cudaSuccess; ++q) {
    if ((t0 + q) % n_sw == 0) {
      e = batch_switch(b->B, b->L, b->st);
      if (e == cudaSuccess) e = batch_colour(b->B, b->L, b->st);
    }
    if (e == cudaSuccess) e = batch_sweep(b->B, b->L, b->st);
    if (e == cudaSuccess) e = batch_step_end(b->B, b->L, b->st);
  }
  return e;
}

// Graph of k steps starting at a step with phase t0 mod n_sw; nullptr if capture fails.
const sco_batch::Graph* get_graph(sco_batch* b, int64_t t0, int k) {
  const int n_sw = b->p[0].n_sw;
  const std::pair<int64_t, int> key(t0 % n_sw, k);
  auto it = b->graphs.find(key);
  if (it != b->graphs.end()) return &it->second;
  const int64_t nl = b->launches;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  const cudaError_t e = enqueue_steps(b, t0, k);
  const cudaError_t e2 = cudaStreamEndCapture(b->st, &g);
  const int64_t captured = b->launches - nl;
  b->launches = nl;  // counted when replayed
  cudaGraphExec_t ex = nullptr;
  if (e == cudaSuccess && e2 == cudaSuccess && g) {
    if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) ex = nullptr;
  }
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  if (!ex) return nullptr;
  auto& slot = b->graphs[key];
  slot.exec = ex;
  slot.launches = captured;
  return &slot;
}

sco_status read_ctl(sco_batch* b) {
  SCO_TRY(cudaMemcpyAsync(b->hctl, b->B.ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, b->st));
  SCO_TRY(cudaStreamSynchronize(b->st));
  if (b->hctl->status != 0 && b->sticky == 0) b->sticky = b->hctl->status;
  return b->sticky ? (sco_status)b->sticky : SCO_OK;
}

// Grows what the flagged step ran out of, clears the flag; the step is then repeated.
sco_status replan(sco_batch* b) {
  BatchDev& B = b->B;
  const BatchCtl& h = *b->hctl;
  SCO_TRY(cudaStreamSynchronize(b->st));
  drop_graphs(b);
  if (h.flag & kReplanCol) {
    const unsigned long long need = h.need_col;
    if (need > 0xFFFFFFFFull) return SCO_ECAPACITY;
    unsigned long long cap = need + need / 4 + 1024;
    if (cap > 0xFFFFFFFFull) cap = 0xFFFFFFFFull;
    cudaFree(B.col);
    B.col = nullptr;
    SCO_TRY(cudaMalloc(&B.col, cap * sizeof(uint32_t)));
    B.col_cap = cap;
  }
  if (h.flag & kReplanOvf) {
    const uint64_t cap = (uint64_t)B.ovf_cap * 2;
    if (cap > 0x7FFFFFFFull) return SCO_ECAPACITY;
    cudaFree(B.ovf);
    B.ovf = nullptr;
    SCO_TRY(cudaMalloc(&B.ovf, 2 * cap * sizeof(uint32_t)));
    B.ovf_cap = (uint32_t)cap;
  }
  if (h.flag & kReplanPal) {
    uint32_t pal = B.pal_cap;
    while (pal < h.gmax + 32 && pal < kPalMax) pal *= 2;
    if (pal > kPalMax) pal = kPalMax;
    if (h.gmax > pal) return SCO_ECAPACITY;
    SCO_TRY(alloc_palette(b, pal));
    set_grids(b);
  }
  SCO_TRY(cudaMemsetAsync(&B.ctl->flag, 0, sizeof(int), b->st));
  SCO_TRY(cudaStreamSynchronize(b->st));
  ++b->replans;
  return SCO_OK;
}

sco_status run_steps(sco_batch* b, int64_t n) {
  if (b->sticky) return (sco_status)b->sticky;
  const int64_t target = b->t + n;
  for (int guard = 0; guard < 64; ++guard) {
    while (b->t < target) {
      const int k = (int)std::min<int64_t>(b->tune.steps_per_graph, target - b->t);
      const sco_batch::Graph* gr = nullptr;
      if (b->tune.use_graph && b->capture_ok) {
        gr = get_graph(b, b->t, k);
        if (!gr) b->capture_ok = false;
      }
      if (gr) {
        SCO_TRY(cudaGraphLaunch(gr->exec, b->st));
        ++b->graph_launches;
        b->launches += gr->launches;
      } else {
        SCO_TRY(enqueue_steps(b, b->t, k));
      }
      b->t += k;
    }
    sco_status s = read_ctl(b);
    if (s != SCO_OK) return s;
    b->t = (int64_t)b->hctl->step;
    if (b->hctl->flag == 0) {
      if (n > 0) b->have_graph = true;
      return SCO_OK;
    }
    s = replan(b);
    if (s != SCO_OK) {
      b->sticky = s;
      return s;
    }
  }
  return SCO_ECAPACITY;
}

bool valid_tuning(const sco_batch_tuning* t) {
  return t && t->steps_per_graph >= 1 && t->steps_per_graph <= 1024 &&
         t->sweep_blocks_per_sm >= 1 && t->kw_blocks_per_sm >= 1 &&
         (t->use_graph == 0 || t->use_graph == 1) && (t->kw_schedule == 0 || t->kw_schedule == 1) &&
         t->kw_low >= 0 && t->kw_low <= 2 &&
         (t->kw_low_group == 1024 || t->kw_low_group == 2048 || t->kw_low_group == 4096);
}

bool same_model(const sco_params& a, const sco_params& b) {
  return a.precision == b.precision && a.n_sw == b.n_sw;
}

}  // namespace

extern "C" {

sco_status sco_batch_init(const sco_params* p, int32_t n, void* stream, sco_batch** out) {
  if (!out) return SCO_EINVAL;
  *out = nullptr;
  if (!p || n < 1 || n > kMaxReplicas) return SCO_EINVAL;
  uint64_t ntot = 0;
  for (int r = 0; r < n; ++r) {
    if (!params_ok(&p[r]) || !same_model(p[0], p[r])) return SCO_EINVAL;
    ntot += (uint64_t)p[r].Lx * p[r].Ly;
  }
  if (ntot >= (1ull << 31)) return SCO_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return SCO_ECUDA;
  sco_batch* b = new (std::nothrow) sco_batch();
  if (!b) return SCO_ENOMEM;
  auto fail = [&](sco_status s) {
    if (b->st) cudaStreamSynchronize(b->st);
    free_all(b);
    delete b;
    return s;
  };
  b->p.assign(p, p + n);
  b->R = n;
  if (stream) {
    b->st = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess)
      return fail(SCO_ECUDA);
    b->own_stream = true;
  }
  BatchDev& B = b->B;
  B.R = n;
  B.Ntot = (uint32_t)ntot;
  B.precision = p[0].precision;
  B.n_sw = p[0].n_sw;
  B.ns_limit = 2000000000ull;
  b->site_start.resize(n + 1);
  b->blk_start.resize(n + 1);
  b->site_start[0] = 0;
  b->blk_start[0] = 0;
  unsigned max_levels = 1;
  for (int r = 0; r < n; ++r) {
    const uint64_t N = (uint64_t)p[r].Lx * p[r].Ly;
    b->site_start[r + 1] = b->site_start[r] + (uint32_t)N;
    b->blk_start[r + 1] = b->blk_start[r] + (uint32_t)((N + kBatchBlock - 1) / kBatchBlock);
    unsigned M = 0;  // levels never exceed ceil(log2 N) (Delta + 1 >= 1)
    while ((1ull << M) < N) ++M;
    max_levels = std::max(max_levels, M);
  }
  B.nblocks = b->blk_start[n];
  B.ntiles = (uint32_t)((ntot + kClassTileSites - 1) / kClassTileSites);
  b->L.levels = max_levels;
  b->L.launches = &b->launches;
  // tables: one sorted list per lattice shape, temperature-dependent tables per replica
  b->P.resize(n);
  b->xy.resize(n);
  b->desc.resize(n);
  std::vector<int> list_of(n, -1);
  std::vector<std::pair<int32_t, int32_t>> shapes;
  for (int r = 0; r < n; ++r) {
    b->P[r] = make_dev_params(p[r]);
    const std::pair<int32_t, int32_t> sh(p[r].Lx, p[r].Ly);
    auto it = std::find(shapes.begin(), shapes.end(), sh);
    if (it == shapes.end()) {
      shapes.push_back(sh);
      b->lists.emplace_back();
      const cudaError_t e = table_build_list(b->P[r], b->lists.back(), b->st, &b->launches);
      if (e != cudaSuccess) return fail(from_cuda(e));
      list_of[r] = (int)shapes.size() - 1;
    } else {
      list_of[r] = (int)(it - shapes.begin());
    }
    const cudaError_t e = table_build_xy(b->P[r], b->xy[r], b->st, &b->launches);
    if (e != cudaSuccess) return fail(from_cuda(e));
    const Table& L = b->lists[list_of[r]];
    RepDesc& d = b->desc[r];
    d.P = b->P[r];
    d.W = L.W;
    d.disp = L.disp;
    d.xy = b->xy[r].xy;
    d.xyq = b->xy[r].xyq;
    d.xy32 = b->xy[r].xy32;
    d.sw64 = b->xy[r].sw64;
    d.sw32 = b->xy[r].sw32;
    d.mnn0 = L.m_nn[0];
    d.mnn1 = L.m_nn[1];
    d.base = b->site_start[r];
    d.variant = p[r].colour_variant;
  }
  const size_t N = ntot;
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc((void**)ptr, bytes > 0 ? bytes : 1);
  };
  RepDesc* d_desc = nullptr;
  uint32_t *d_blk = nullptr, *d_site = nullptr;
  A(&d_desc, n * sizeof(RepDesc));
  A(&d_blk, (n + 1) * sizeof(uint32_t));
  A(&d_site, (n + 1) * sizeof(uint32_t));
  B.desc = d_desc;
  B.blk_start = d_blk;
  B.site_start = d_site;
  A(&B.plan, n * sizeof(RepPlan));
  A(&B.cnt, n * sizeof(DevCounters));
  A(&B.ctl, sizeof(BatchCtl));
  A(&B.s, 3 * N * sizeof(double));
  A(&B.s32, N * sizeof(float4));
  A(&B.acc, N);
  A(&B.hslot, N * kSlotCap * sizeof(uint32_t));
  A(&B.hcnt, N * sizeof(uint32_t));
  A(&B.indeg, N * sizeof(uint32_t));
  A(&B.deg, (N + 1) * sizeof(uint32_t));
  A(&B.lcur, N * sizeof(uint32_t));
  A(&B.ocur, N * sizeof(uint32_t));
  B.ovf_cap = (uint32_t)std::max<size_t>(N, 65536);
  A(&B.ovf, 2 * (size_t)B.ovf_cap * sizeof(uint32_t));
  A(&B.row_ptr, (N + 1) * sizeof(uint32_t));
  B.col_cap = (unsigned long long)N * 24 + 1024;
  A(&B.col, B.col_cap * sizeof(uint32_t));
  A(&B.word, N * sizeof(unsigned long long));
  A(&B.col8, N);
  A(&B.blk, N * sizeof(uint32_t));
  A(&B.colour, N * sizeof(uint32_t));
  A(&B.perm, N * sizeof(uint32_t));
  A(&B.defer, N * sizeof(uint32_t));
  A(&B.prop, N * sizeof(double4_32a));
  A(&B.imask, N * sizeof(unsigned long long));
  A(&B.imeta, N * sizeof(uint32_t));
  A(&B.ilist, kKwItemList * N * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMallocHost(&b->hcnt, n * sizeof(DevCounters));
  if (e == cudaSuccess) e = cudaMallocHost(&b->hctl, sizeof(BatchCtl));
  if (e == cudaSuccess) e = alloc_palette(b, 256);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_desc, b->desc.data(), n * sizeof(RepDesc), cudaMemcpyHostToDevice, b->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_blk, b->blk_start.data(), (n + 1) * sizeof(uint32_t),
                        cudaMemcpyHostToDevice, b->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_site, b->site_start.data(), (n + 1) * sizeof(uint32_t),
                        cudaMemcpyHostToDevice, b->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(B.cnt, 0, n * sizeof(DevCounters), b->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(B.ctl, 0, sizeof(BatchCtl), b->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(B.deg, 0, (N + 1) * sizeof(uint32_t), b->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(B.acc, 0, N, b->st);
  for (int r = 0; r < n && e == cudaSuccess; ++r) {
    const size_t so = 3 * (size_t)b->site_start[r];
    e = spins_init(b->P[r], B.s + so, B.s32 + b->site_start[r], b->st, &b->launches);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return fail(from_cuda(e));
  b->tune.kw_schedule = 0;
  b->tune.kw_low = 1;
  b->tune.kw_low_group = 2048;
  b->kw_occ = batch_kw_occupancy(0, n, B.pal_cap);
  b->sweep_occ = batch_sweep_occupancy(B.precision, n);
  b->tune.steps_per_graph = 4;
  b->tune.sweep_blocks_per_sm = b->sweep_occ;
  b->tune.kw_blocks_per_sm = std::min(4, b->kw_occ);
  b->tune.use_graph = 1;
  set_grids(b);
  *out = b;
  return SCO_OK;
}

void sco_batch_destroy(sco_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->st);
  free_all(b);
  delete b;
}

sco_status sco_batch_run(sco_batch* b, int32_t n_mcs) {
  if (!b || n_mcs < 0) return SCO_EINVAL;
  return run_steps(b, n_mcs);
}

sco_status sco_batch_set_tuning(sco_batch* b, const sco_batch_tuning* t) {
  if (!b || !valid_tuning(t)) return SCO_EINVAL;
  SCO_TRY(cudaStreamSynchronize(b->st));
  const bool grids = t->sweep_blocks_per_sm != b->tune.sweep_blocks_per_sm ||
                     t->kw_blocks_per_sm != b->tune.kw_blocks_per_sm ||
                     t->kw_schedule != b->tune.kw_schedule || t->kw_low != b->tune.kw_low ||
                     t->kw_low_group != b->tune.kw_low_group;
  b->tune = *t;
  b->tune.sweep_blocks_per_sm = std::min(t->sweep_blocks_per_sm, b->sweep_occ);
  if (grids) drop_graphs(b);
  set_grids(b);
  b->tune.kw_blocks_per_sm = std::min(t->kw_blocks_per_sm, b->kw_occ);
  return SCO_OK;
}

sco_status sco_batch_get_tuning(sco_batch* b, sco_batch_tuning* t) {
  if (!b || !t) return SCO_EINVAL;
  *t = b->tune;
  return SCO_OK;
}

sco_status sco_batch_autotune(sco_batch* b, int32_t trial, sco_batch_tuning* chosen) {
  if (!b || trial < 1) return SCO_EINVAL;
  if (b->sticky) return (sco_status)b->sticky;
  // one step first: buffers settle (a replan, if any, happens here)
  sco_status s = run_steps(b, 1);
  if (s != SCO_OK) return s;
  cudaEvent_t ea = nullptr, eb = nullptr;
  SCO_TRY(cudaEventCreate(&ea));
  SCO_TRY(cudaEventCreate(&eb));
  auto time_of = [&](const sco_batch_tuning& t, double& ms) -> sco_status {
    sco_status st = sco_batch_set_tuning(b, &t);
    if (st == SCO_OK) st = run_steps(b, t.steps_per_graph);  // warm-up (captures the graph)
    if (st != SCO_OK) return st;
    const int32_t k = std::max(trial, t.steps_per_graph);
    if (cudaEventRecord(ea, b->st) != cudaSuccess) return SCO_ECUDA;
    st = run_steps(b, k);
    if (st != SCO_OK) return st;
    if (cudaEventRecord(eb, b->st) != cudaSuccess || cudaEventSynchronize(eb) != cudaSuccess)
      return SCO_ECUDA;
    float f = 0.f;
    if (cudaEventElapsedTime(&f, ea, eb) != cudaSuccess) return SCO_ECUDA;
    ms = f / k;
    return SCO_OK;
  };
  sco_batch_tuning best = b->tune;
  double best_ms = 0.0;
  s = time_of(best, best_ms);
  auto try_dim = [&](std::vector<sco_batch_tuning> cands) {
    for (const auto& c : cands) {
      if (s != SCO_OK) return;
      double ms = 0.0;
      s = time_of(c, ms);
      if (s == SCO_OK && ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
  };
  {
    std::vector<sco_batch_tuning> c;
    for (int v : {1, 2, 3, 4, 6, 8})
      if (v <= b->sweep_occ && v != best.sweep_blocks_per_sm) {
        sco_batch_tuning t = best;
        t.sweep_blocks_per_sm = v;
        c.push_back(t);
      }
    try_dim(c);
  }
  {
    sco_batch_tuning t = best;
    t.kw_schedule = 1 - best.kw_schedule;
    try_dim({t});
  }
  {
    std::vector<sco_batch_tuning> c;
    for (int v : {1024, 2048, 4096})
      if (v != best.kw_low_group || best.kw_low != 1) {
        sco_batch_tuning t = best;
        t.kw_low = 1;
        t.kw_low_group = v;
        c.push_back(t);
      }
    if (best.kw_low != 0) {
      sco_batch_tuning t = best;
      t.kw_low = 0;
      c.push_back(t);
    }
    try_dim(c);
  }
  {
    std::vector<sco_batch_tuning> c;
    for (int v : {1, 2, 4})
      if (v != best.kw_blocks_per_sm) {
        sco_batch_tuning t = best;
        t.kw_blocks_per_sm = v;
        c.push_back(t);
      }
    try_dim(c);
  }
  {
    std::vector<sco_batch_tuning> c;
    for (int v : {1, 2, 8, 16})
      if (v != best.steps_per_graph) {
        sco_batch_tuning t = best;
        t.steps_per_graph = v;
        c.push_back(t);
      }
    sco_batch_tuning t = best;
    t.use_graph = 0;
    t.steps_per_graph = 1;
    c.push_back(t);
    try_dim(c);
  }
  cudaEventDestroy(ea);
  cudaEventDestroy(eb);
  if (s != SCO_OK) return s;
  s = sco_batch_set_tuning(b, &best);
  if (s == SCO_OK && chosen) *chosen = best;
  return s;
}

sco_status sco_batch_observables(sco_batch* b, int32_t r, sco_obs* o, int32_t want_full) {
  if (!b || !o || r < 0 || r >= b->R) return SCO_EINVAL;
  if (b->sticky) return (sco_status)b->sticky;
  const DevParams& P = b->P[r];
  const uint32_t base = b->site_start[r];
  const bool full = want_full && P.N <= 65536;
  SCO_TRY(observables_run(P, b->B.s + 3 * (size_t)base, b->B.row_ptr + base, b->B.col,
                          b->xy[r].xy, b->have_graph, full, b->B.cnt + r, b->st, &b->launches));
  SCO_TRY(cudaMemcpyAsync(b->hcnt + r, b->B.cnt + r, sizeof(DevCounters), cudaMemcpyDeviceToHost,
                          b->st));
  sco_status s = read_ctl(b);
  if (s != SCO_OK) return s;
  const DevCounters& h = b->hcnt[r];
  const double N = (double)P.N;
  std::memset(o, 0, sizeof(*o));
  const bool g = b->have_graph;
  o->e_exchange = h.acc[4];
  o->e_switched = (g ? h.acc[5] : 0.0) + h.acc[4];
  o->e_full = full ? h.acc[6] : NAN;
  o->mx = h.acc[0] / N;
  o->my = h.acc[1] / N;
  o->mz = h.acc[2] / N;
  o->m_abs = std::sqrt(o->mx * o->mx + o->my * o->my + o->mz * o->mz);
  o->m_phi = h.acc[3] / N;
  o->n_edges = g ? (int64_t)h.n_dip : 0;
  o->max_degree = g ? (int32_t)h.max_degree : 0;
  o->max_degree_dipolar = g ? (int32_t)h.max_degree_dip : 0;
  o->n_colours = g ? (int32_t)h.n_colours : 0;
  o->kw_rounds = g ? (int32_t)h.kw_rounds : 0;
  o->sweeps_done = b->t;
  o->guard_hits_fp64 = (int64_t)h.guard_fp64;
  o->guard_hits_fp32 = (int64_t)h.guard_fp32;
  o->kernel_launches = b->launches;
  return SCO_OK;
}

sco_status sco_batch_get_spins(sco_batch* b, int32_t r, double* xyz, int32_t on_device) {
  if (!b || !xyz || r < 0 || r >= b->R) return SCO_EINVAL;
  const size_t N = (size_t)b->P[r].N;
  SCO_TRY(cudaMemcpyAsync(xyz, b->B.s + 3 * (size_t)b->site_start[r], 3 * N * sizeof(double),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->st));
  SCO_TRY(cudaStreamSynchronize(b->st));
  return b->sticky ? (sco_status)b->sticky : SCO_OK;
}

sco_status sco_batch_set_spins(sco_batch* b, int32_t r, const double* xyz, int32_t on_device) {
  if (!b || !xyz || r < 0 || r >= b->R) return SCO_EINVAL;
  const size_t N = (size_t)b->P[r].N, so = 3 * (size_t)b->site_start[r];
  SCO_TRY(cudaMemcpyAsync(b->B.s + so, xyz, 3 * N * sizeof(double),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->st));
  SCO_TRY(spins_to_f32((int64_t)N, b->B.s + so, b->B.s32 + b->site_start[r], b->st,
                       &b->launches));
  SCO_TRY(cudaStreamSynchronize(b->st));
  return SCO_OK;
}

sco_status sco_batch_get_sizes(sco_batch* b, int32_t r, int64_t* n_sites, int64_t* n_entries,
                               int32_t* max_degree, int32_t* palette) {
  if (!b || r < 0 || r >= b->R) return SCO_EINVAL;
  SCO_TRY(cudaMemcpyAsync(b->hcnt + r, b->B.cnt + r, sizeof(DevCounters), cudaMemcpyDeviceToHost,
                          b->st));
  SCO_TRY(cudaStreamSynchronize(b->st));
  const DevCounters& h = b->hcnt[r];
  const bool g = b->have_graph;
  if (n_sites) *n_sites = b->P[r].N;
  if (n_entries) *n_entries = g ? (int64_t)h.nnz : 0;
  if (max_degree) *max_degree = g ? (int32_t)h.max_degree : 0;
  if (palette) *palette = g ? (int32_t)h.g : 0;
  return SCO_OK;
}

sco_status sco_batch_get_graph(sco_batch* b, int32_t r, uint32_t* row_ptr, uint32_t* col,
                               uint32_t* colour) {
  if (!b || r < 0 || r >= b->R) return SCO_EINVAL;
  if (!b->have_graph) return SCO_ESTATE;
  const uint32_t base = b->site_start[r];
  const size_t N = (size_t)b->P[r].N;
  std::vector<uint32_t> rp(N + 1);
  SCO_TRY(cudaMemcpyAsync(rp.data(), b->B.row_ptr + base, (N + 1) * sizeof(uint32_t),
                          cudaMemcpyDeviceToHost, b->st));
  SCO_TRY(cudaStreamSynchronize(b->st));
  const uint32_t e0 = rp[0];
  if (row_ptr)
    for (size_t i = 0; i <= N; ++i) row_ptr[i] = rp[i] - e0;
  if (col && rp[N] > e0)
    SCO_TRY(cudaMemcpyAsync(col, b->B.col + e0, (size_t)(rp[N] - e0) * sizeof(uint32_t),
                            cudaMemcpyDeviceToHost, b->st));
  if (colour)
    SCO_TRY(cudaMemcpyAsync(colour, b->B.colour + base, N * sizeof(uint32_t),
                            cudaMemcpyDeviceToHost, b->st));
  return read_ctl(b);
}

sco_status sco_batch_get_accepts(sco_batch* b, int32_t r, uint8_t* acc) {
  if (!b || !acc || r < 0 || r >= b->R) return SCO_EINVAL;
  SCO_TRY(cudaMemcpyAsync(acc, b->B.acc + b->site_start[r], (size_t)b->P[r].N,
                          cudaMemcpyDeviceToHost, b->st));
  return read_ctl(b);
}

sco_status sco_batch_info(sco_batch* b, int64_t* total_sites, int64_t* steps_done,
                          int64_t* launches, int64_t* graph_launches, int32_t* replans) {
  if (!b) return SCO_EINVAL;
  if (total_sites) *total_sites = b->B.Ntot;
  if (steps_done) *steps_done = b->t;
  if (launches) *launches = b->launches;
  if (graph_launches) *graph_launches = b->graph_launches;
  if (replans) *replans = b->replans;
  return SCO_OK;
}

sco_status sco_batch_sync(sco_batch* b) {
  if (!b) return SCO_EINVAL;
  return read_ctl(b);
}

sco_status sco_batch_set_temperature(sco_batch* b, int32_t r, double T) {
  if (!b || r < 0 || r >= b->R) return SCO_EINVAL;
  if (b->sticky) return (sco_status)b->sticky;
  sco_params q = b->p[r];
  q.T = T;
  if (!params_ok(&q)) return SCO_EINVAL;
  // every replica switches at the steps t with t mod n_sw = 0: a change there takes effect with
  // that switch, so the replica's graph never mixes two temperatures
  if (b->t % b->B.n_sw != 0) return SCO_ESTATE;
  SCO_TRY(cudaStreamSynchronize(b->st));
  drop_graphs(b);
  b->p[r] = q;
  b->P[r] = make_dev_params(q);
  table_free_xy(b->xy[r]);
  SCO_TRY(table_build_xy(b->P[r], b->xy[r], b->st, &b->launches));
  RepDesc& d = b->desc[r];
  d.P = b->P[r];
  d.xy = b->xy[r].xy;
  d.xyq = b->xy[r].xyq;
  d.xy32 = b->xy[r].xy32;
  d.sw64 = b->xy[r].sw64;
  d.sw32 = b->xy[r].sw32;
  SCO_TRY(cudaMemcpyAsync(const_cast<RepDesc*>(b->B.desc) + r, &d, sizeof(RepDesc),
                          cudaMemcpyHostToDevice, b->st));
  SCO_TRY(cudaStreamSynchronize(b->st));
  return SCO_OK;
}

sco_status sco_batch_set_wait_limit(sco_batch* b, uint64_t ns) {
  if (!b || ns > 3600000000000ull) return SCO_EINVAL;
  SCO_TRY(cudaStreamSynchronize(b->st));
  b->B.ns_limit = ns;
  drop_graphs(b);  // captured launches hold the old limit
  return SCO_OK;
}

}  // extern "C"
