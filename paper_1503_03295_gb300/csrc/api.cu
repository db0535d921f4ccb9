// api.cu -- the C ABI (include/sco.h): context lifetime, the per-step schedule of Fig. 1
// (switch -> colour -> colour-class sweeps), getters, checkpoints and phase timing.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "sco.h"
#include "sco_internal.h"
#include "batch.h"

namespace sco {

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      n = 1;
  }
  return n;
}

// ln 2 = 2 atanh(1/3) = 2 sum_k 3^-(2k+1) / (2k+1), summed in double-double.
static dd ln2_dd() {
  const dd third = dd_div(dd_from(1.0), dd_from(3.0));
  const dd x2 = dd_mul(third, third);
  dd pw = third, sum = dd_from(0.0);
  for (int k = 0; k < 40; ++k) {
    sum = dd_add(sum, dd_div(pw, dd_from(2.0 * k + 1.0)));
    pw = dd_mul(pw, x2);
  }
  return dd_ldexp(sum, 1);
}

bool params_ok(const sco_params* p) {
  if (!p) return false;
  if (p->Lx < 1 || p->Ly < 1 || p->Lx > 32767 || p->Ly > 32767) return false;
  if ((int64_t)p->Lx * p->Ly >= (1ll << 30)) return false;
  if (!(p->T > 0.0) || !std::isfinite(p->T) || !(p->D >= 0.0) || !std::isfinite(p->D) ||
      !std::isfinite(p->J))
    return false;
  if (p->n_sw < 1 || p->precision < 0 || p->precision > 1) return false;
  if (p->colour_variant < 0 || p->colour_variant > 1) return false;
  return true;
}


DevParams make_dev_params(const sco_params& p) {
  DevParams P{};
  P.Lx = p.Lx;
  P.Ly = p.Ly;
  P.N = (int64_t)p.Lx * p.Ly;
  P.K = (int64_t)(p.Lx - 1) + (int64_t)(p.Ly - 1) * (2 * (int64_t)p.Lx - 1);
  P.J = p.J;
  P.D = p.D;
  P.beta = 1.0 / p.T;
  P.bD = P.beta * p.D;
  P.inv_bD58 = P.bD > 0.0 ? 0x1p58 / P.bD : 0.0;
  P.inv_bD58_f = (float)P.inv_bD58;
  P.beta_f = (float)P.beta;
  P.bJ_f = (float)(P.beta * P.J);
  P.switching = P.bD > 0.0 ? 1 : 0;
  P.lx_magic = div_magic((unsigned long long)p.Lx);
  P.key0 = p.seed;
  P.key1 = (uint64_t)(uint32_t)p.replica;
  const dd l2 = ln2_dd();
  P.ln2_hi = l2.hi;
  P.ln2_lo = l2.lo;
  return P;
}

}  // namespace sco

using namespace sco;

namespace {

enum Phase { kPhSwitch = 0, kPhColour = 1, kPhSweep = 2 };

struct StateHeader {
  char magic[8];
  uint32_t version;
  uint32_t has_epoch;
  sco_params p;
  int64_t t;
  int64_t N;
};

}  // namespace

struct sco_ctx {
  sco_params p{};
  DevParams P{};
  cudaStream_t st = nullptr;
  int64_t launches = 0;
  Table tab;
  double* s = nullptr;
  float4* s32 = nullptr;  // FP32 copy of the spins, one (x, y, z, 0) per site
  double* s_epoch = nullptr;
  SwitchBufs sw{};
  uint32_t* row_ptr = nullptr;
  uint32_t* col = nullptr;
  uint64_t col_cap = 0;
  ColourBufs cb{};
  uint32_t cls_cap = 0;  // capacity of hist / off / cursor
  uint8_t* acc = nullptr;
  uint32_t* defer = nullptr;  // N sites whose decision goes to the warp-parallel resolve
  double4_32a* prop = nullptr;  // N proposals {S', u} of the current MC step
  DevCounters* cnt = nullptr;   // device
  DevCounters* hcnt = nullptr;  // pinned mirror
  int64_t t = 0;
  int64_t graph_epoch = -1;
  bool colour_valid = false;
  uint32_t g = 1;
  uint64_t nnz = 0;
  // FP64 form: the pair cache (hid parallel to col, keep records in SwitchBufs, upd per site);
  // cache_state 0: the first halves hold the terms at the current spins; 1: the halves given by
  // the parities of the last step hold them; 2: rebuild from the spins first
  uint32_t* hid = nullptr;
  uint8_t* upd = nullptr;
  int cache_state = 0;
  bool dip_valid = false;  // cnt->max_degree_dip holds the dipolar Delta of the current graph
  int sticky = 0;
  unsigned long long ns_limit = 2000000000ull;  // bound of every device-side wait (2 s)
  // phase timing
  bool timing = false;
  struct Ev {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<Ev> evs;
  std::vector<cudaEvent_t> pool;
  double ms[3] = {0, 0, 0};
  int64_t calls[3] = {0, 0, 0};
};

namespace {

sco_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return SCO_OK;
  if (e == cudaErrorMemoryAllocation) return SCO_ENOMEM;
  return SCO_ECUDA;
}

#define SCO_TRY(expr)                                \
  do {                                               \
    const cudaError_t e_ = (expr);                   \
    if (e_ != cudaSuccess) return from_cuda(e_);     \
  } while (0)

cudaEvent_t take_event(sco_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

struct PhaseTimer {
  sco_ctx* c;
  int phase;
  cudaEvent_t a = nullptr;
  PhaseTimer(sco_ctx* cc, int ph) : c(cc), phase(ph) {
    if (c->timing) {
      a = take_event(c);
      cudaEventRecord(a, c->st);
    }
  }
  ~PhaseTimer() {
    if (c->timing && a) {
      cudaEvent_t b = take_event(c);
      cudaEventRecord(b, c->st);
      c->evs.push_back({phase, a, b});
    }
  }
};

sco_status read_counters(sco_ctx* c) {
  SCO_TRY(cudaMemcpyAsync(c->hcnt, c->cnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, c->st));
  SCO_TRY(cudaStreamSynchronize(c->st));
  if (c->hcnt->status != 0 && c->sticky == 0) c->sticky = c->hcnt->status;
  return c->sticky ? (sco_status)c->sticky : SCO_OK;
}

template <typename T>
cudaError_t grow(T*& ptr, uint64_t& cap, uint64_t need) {
  if (need <= cap && ptr) return cudaSuccess;
  uint64_t ncap = need + need / 4 + 1024;
  cudaFree(ptr);
  ptr = nullptr;
  cap = 0;
  cudaError_t e = cudaMalloc(&ptr, ncap * sizeof(T));
  if (e == cudaSuccess) cap = ncap;
  return e;
}

bool cache_on(const sco_ctx* c) { return c->sw.keep != nullptr; }

// The per-half-edge records of the pair cache for the current overflow capacity.
cudaError_t alloc_keep(sco_ctx* c) {
  cudaFree(c->sw.keep);
  c->sw.keep = nullptr;
  const size_t n = (size_t)c->P.N * kSlotCap + c->sw.ovf_cap;
  return cudaMalloc(&c->sw.keep, n * sizeof(double4_32a));
}

PairCache pair_cache(sco_ctx* c) {
  if (!cache_on(c)) return PairCache{};
  // the last endpoint's term is needed only when the next step keeps this graph
  const int carry = (c->t + 1) % c->p.n_sw != 0 ? 1 : 0;
  return PairCache{c->hid, c->sw.keep, c->upd, carry, c->cache_state != 1 ? 1 : 0};
}

sco_status do_switch(sco_ctx* c, uint32_t epoch, const double* src, const float4* src32) {
  PhaseTimer tm(c, kPhSwitch);
  // per-switch counters: n_half, n_dip, ovf_n, nnz and max_degree, max_degree_dip
  SCO_TRY(cudaMemsetAsync(c->cnt, 0, 4 * sizeof(unsigned long long), c->st));
  SCO_TRY(cudaMemsetAsync(&c->cnt->max_degree, 0, 2 * sizeof(unsigned), c->st));
  if (c->p.n_sw > 1 && src == c->s)
    SCO_TRY(cudaMemcpyAsync(c->s_epoch, c->s, 3 * c->P.N * sizeof(double),
                            cudaMemcpyDeviceToDevice, c->st));
  SCO_TRY(switch_run(c->P, c->tab, src, src32, c->p.precision, epoch, c->sw, c->cnt, c->st,
                     &c->launches));
  SCO_TRY(csr_scan(c->P, c->sw, c->row_ptr, c->cnt, c->st, &c->launches));
  sco_status st = read_counters(c);
  if (st != SCO_OK) return st;
  if (c->hcnt->ovf_n > c->sw.ovf_cap) {
    // more half-edges beyond the per-site slots than the overflow list holds: grow it and
    // switch again (the switch is a pure function of the spins and the epoch)
    const unsigned long long need = c->hcnt->ovf_n + c->hcnt->ovf_n / 4 + 1024;
    if (need > 0x7FFFFFFFull) return SCO_ECAPACITY;
    cudaFree(c->sw.ovf);
    c->sw.ovf = nullptr;
    SCO_TRY(cudaMalloc(&c->sw.ovf, 2 * need * sizeof(uint32_t)));
    c->sw.ovf_cap = (uint32_t)need;
    if (cache_on(c)) {
      // half-edge ids must stay below 2^32 for the cache: else run without it
      if ((uint64_t)c->P.N * kSlotCap + need >= (1ull << 32)) {
        cudaFree(c->sw.keep);
        c->sw.keep = nullptr;
        cudaFree(c->hid);
        c->hid = nullptr;
      } else {
        SCO_TRY(alloc_keep(c));
      }
    }
    SCO_TRY(cudaMemsetAsync(c->cnt, 0, 4 * sizeof(unsigned long long), c->st));
    SCO_TRY(cudaMemsetAsync(&c->cnt->max_degree, 0, 2 * sizeof(unsigned), c->st));
    SCO_TRY(cudaMemsetAsync(&c->cnt->ovf_full, 0, sizeof(int), c->st));
    SCO_TRY(switch_run(c->P, c->tab, src, src32, c->p.precision, epoch, c->sw, c->cnt, c->st,
                       &c->launches));
    SCO_TRY(csr_scan(c->P, c->sw, c->row_ptr, c->cnt, c->st, &c->launches));
    st = read_counters(c);
    if (st != SCO_OK) return st;
    if (c->hcnt->ovf_n > c->sw.ovf_cap) return SCO_ECAPACITY;
  }
  c->nnz = c->hcnt->nnz;
  if (c->col_cap < c->nnz) {
    cudaFree(c->hid);
    c->hid = nullptr;
  }
  SCO_TRY(grow(c->col, c->col_cap, c->nnz > 0 ? c->nnz : 1));
  if (cache_on(c) && !c->hid) SCO_TRY(cudaMalloc(&c->hid, c->col_cap * sizeof(uint32_t)));
  // rows are left unsorted (their order changes no result); getters sort their copies
  SCO_TRY(csr_fill(c->P, c->sw, c->row_ptr, c->col, cache_on(c) ? c->hid : nullptr,
                   c->hcnt->ovf_n > 0, false, c->cnt, c->st, &c->launches));
  c->dip_valid = false;
  // the switch left the FP64 terms of the switching spins in the cache: valid now unless the
  // graph was switched from other spins (the epoch start of a restored checkpoint)
  c->cache_state = src == c->s ? 0 : 2;
  c->g = c->hcnt->max_degree + 1;
  c->graph_epoch = epoch;
  c->colour_valid = false;
  return SCO_OK;
}

sco_status do_colour(sco_ctx* c) {
  PhaseTimer tm(c, kPhColour);
  if (c->g + 1 > c->cls_cap) {
    cudaFree(c->cb.hist);
    cudaFree(c->cb.off);
    cudaFree(c->cb.cursor);
    cudaFree(c->cb.scan_tmp);
    cudaFree(c->cb.tile_cnt);
    cudaFree(c->cb.dcnt);
    cudaFree(c->cb.bcnt);
    c->cb.hist = c->cb.off = c->cb.cursor = c->cb.tile_cnt = c->cb.dcnt = c->cb.bcnt = nullptr;
    c->cb.scan_tmp = nullptr;
    const uint32_t cap = c->g + 64;
    const int64_t ntiles = (c->P.N + kClassTileSites - 1) / kClassTileSites;
    // (colour, degree bin) keys per tile: at most max(palette, 8192) (see bucket_run)
    const int64_t keys = cap < kMaxStablePalette ? cap : kMaxStablePalette;
    const int64_t tc = (keys > 8192 ? keys : 8192) * ntiles + 1;
    SCO_TRY(cudaMalloc(&c->cb.hist, (cap + 1) * sizeof(uint32_t)));
    SCO_TRY(cudaMalloc(&c->cb.off, (cap + 1) * sizeof(uint32_t)));
    SCO_TRY(cudaMalloc(&c->cb.cursor, (cap + 1) * sizeof(uint32_t)));
    SCO_TRY(cudaMalloc(&c->cb.dcnt, (cap + 1) * sizeof(uint32_t)));
    SCO_TRY(cudaMalloc(&c->cb.bcnt, (size_t)32 * (cap + 1) * sizeof(uint32_t)));
    if (!c->cb.boff) SCO_TRY(cudaMalloc(&c->cb.boff, (size_t)kKwSplitBlocks * 64 * sizeof(uint32_t)));
    SCO_TRY(cudaMalloc(&c->cb.tile_cnt, tc * sizeof(uint32_t)));
    SCO_TRY(cudaMalloc(&c->cb.scan_tmp, scan_tmp_bytes(tc > cap + 1 ? tc : cap + 1)));
    c->cls_cap = cap;
  }
  SCO_TRY(kw_run(c->P, c->row_ptr, c->col, c->g, c->p.colour_variant, c->cb, c->cnt,
                 c->ns_limit, c->st, &c->launches));
  SCO_TRY(bucket_run(c->P, c->g, c->row_ptr, c->cb, c->cnt, c->st, &c->launches));
  c->colour_valid = true;
  return SCO_OK;
}

sco_status ensure_graph(sco_ctx* c) {
  const int64_t e = c->t / c->p.n_sw;
  if (c->graph_epoch != e) {
    sco_status st = do_switch(c, (uint32_t)e, c->s, c->s32);
    if (st != SCO_OK) return st;
  }
  if (!c->colour_valid) return do_colour(c);
  return SCO_OK;
}

void free_all(sco_ctx* c) {
  table_free(c->tab);
  cudaFree(c->s);
  cudaFree(c->s32);
  cudaFree(c->s_epoch);
  cudaFree(c->sw.hslot);
  cudaFree(c->sw.hcnt);
  cudaFree(c->sw.indeg);
  cudaFree(c->sw.deg);
  cudaFree(c->sw.lcur);
  cudaFree(c->sw.ocur);
  cudaFree(c->sw.ovf);
  cudaFree(c->sw.scan_tmp);
  cudaFree(c->sw.keep);
  cudaFree(c->hid);
  cudaFree(c->upd);
  cudaFree(c->row_ptr);
  cudaFree(c->col);
  cudaFree(c->cb.word);
  cudaFree(c->cb.col8);
  cudaFree(c->cb.blk);
  cudaFree(c->cb.colour);
  cudaFree(c->cb.hist);
  cudaFree(c->cb.off);
  cudaFree(c->cb.cursor);
  cudaFree(c->cb.perm);
  cudaFree(c->cb.tile_cnt);
  cudaFree(c->cb.scan_tmp);
  cudaFree(c->cb.bcnt);
  cudaFree(c->cb.boff);
  cudaFree(c->cb.meta);
  cudaFree(c->cb.imask);
  cudaFree(c->cb.imeta);
  cudaFree(c->cb.ilist);
  cudaFree(c->acc);
  cudaFree(c->defer);
  cudaFree(c->prop);
  cudaFree(c->cnt);
  if (c->hcnt) cudaFreeHost(c->hcnt);
  for (auto& e : c->evs) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
}

}  // namespace

extern "C" {

const char* sco_strerror(sco_status s) {
  switch (s) {
    case SCO_OK: return "ok";
    case SCO_EINVAL: return "invalid argument";
    case SCO_ENOMEM: return "device allocation failed";
    case SCO_ECUDA: return "CUDA runtime error";
    case SCO_ETIMEOUT: return "bounded device wait gave up";
    case SCO_ESTATE: return "invalid state";
    case SCO_EGUARD: return "guard failure";
    case SCO_ECAPACITY: return "device buffer capacity exceeded";
  }
  return "unknown status";
}

sco_status sco_init(const sco_params* p, void* stream, sco_ctx** out) {
  if (!out) return SCO_EINVAL;
  *out = nullptr;
  if (!params_ok(p)) return SCO_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return SCO_ECUDA;
  sco_ctx* c = new (std::nothrow) sco_ctx();
  if (!c) return SCO_ENOMEM;
  c->p = *p;
  c->st = (cudaStream_t)stream;
  c->P = make_dev_params(*p);
  const DevParams& P = c->P;
  const int64_t N = P.N;
  auto fail = [&](sco_status s) {
    free_all(c);
    delete c;
    return s;
  };
  cudaError_t e = table_build(P, c->tab, c->st, &c->launches);
  if (e != cudaSuccess) return fail(from_cuda(e));
  e = cudaMalloc(&c->s, 3 * N * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->s32, N * sizeof(float4));
  if (e == cudaSuccess && p->n_sw > 1) e = cudaMalloc(&c->s_epoch, 3 * N * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->sw.hslot, N * kSlotCap * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&c->sw.hcnt, N * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&c->sw.indeg, N * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&c->sw.deg, (N + 1) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&c->sw.lcur, N * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&c->sw.ocur, N * sizeof(uint32_t));
  c->sw.ovf_cap = (uint32_t)(N > 65536 ? N : 65536);
  if (e == cudaSuccess) e = cudaMalloc(&c->sw.ovf, 2 * (size_t)c->sw.ovf_cap * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&c->sw.scan_tmp, scan_tmp_bytes(N + 1));
  if (e == cudaSuccess) e = cudaMalloc(&c->row_ptr, (N + 1) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&c->cb.word, N * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&c->cb.col8, N);
  if (e == cudaSuccess) e = cudaMalloc(&c->cb.blk, N * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&c->cb.colour, N * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&c->cb.perm, N * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&c->cb.meta, 8 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&c->cb.imask, N * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&c->cb.imeta, N * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&c->cb.ilist, kKwItemList * N * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&c->acc, N);
  if (e == cudaSuccess) e = cudaMalloc(&c->defer, N * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&c->prop, N * sizeof(double4_32a));
  if (e == cudaSuccess) e = cudaMalloc(&c->cnt, sizeof(DevCounters));
  if (e == cudaSuccess) e = cudaMallocHost(&c->hcnt, sizeof(DevCounters));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->cnt, 0, sizeof(DevCounters), c->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->acc, 0, N, c->st);
  if (e != cudaSuccess) return fail(from_cuda(e));
  // the FP64 form keeps the pair cache while half-edge ids fit 32 bits
  if (p->precision == SCO_FP64 && (uint64_t)N * kSlotCap + c->sw.ovf_cap < (1ull << 32)) {
    e = alloc_keep(c);
    if (e == cudaSuccess) e = cudaMalloc(&c->upd, N);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->upd, 0, N, c->st);
    if (e != cudaSuccess) return fail(from_cuda(e));
  }
  const uint64_t guess = (uint64_t)N * 24 + 1024;
  e = grow(c->col, c->col_cap, guess);
  if (e == cudaSuccess) e = spins_init(P, c->s, c->s32, c->st, &c->launches);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return fail(from_cuda(e));
  *out = c;
  return SCO_OK;
}

void sco_destroy(sco_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  free_all(c);
  delete c;
}

sco_status sco_switch(sco_ctx* c) {
  if (!c) return SCO_EINVAL;
  if (c->sticky) return (sco_status)c->sticky;
  return do_switch(c, (uint32_t)(c->t / c->p.n_sw), c->s, c->s32);
}

sco_status sco_colour(sco_ctx* c, int32_t* n_colours) {
  if (!c) return SCO_EINVAL;
  if (c->sticky) return (sco_status)c->sticky;
  sco_status st = SCO_OK;
  if (c->graph_epoch < 0) st = sco_switch(c);
  if (st == SCO_OK) st = do_colour(c);
  if (st == SCO_OK && n_colours) {
    st = read_counters(c);
    *n_colours = (int32_t)c->hcnt->n_colours;
  }
  return st;
}

sco_status sco_sweep(sco_ctx* c, int32_t n_mcs) {
  if (!c || n_mcs < 0) return SCO_EINVAL;
  if (c->sticky) return (sco_status)c->sticky;
  for (int32_t k = 0; k < n_mcs; ++k) {
    sco_status st = ensure_graph(c);
    if (st != SCO_OK) return st;
    {
      PhaseTimer tm(c, kPhSweep);
      if (cache_on(c) && c->cache_state == 2)
        SCO_TRY(cache_build_run(c->P, c->tab, c->s, c->sw, c->cnt, c->st, &c->launches));
      SCO_TRY(sweep_run(c->P, c->tab, c->s, c->s32, c->row_ptr, c->col, c->cb.perm, c->cb.off,
                        c->g, (uint64_t)c->t, c->p.precision, c->acc, c->defer, c->cb.dcnt,
                        c->prop, c->cnt, pair_cache(c), c->st, &c->launches));
      c->cache_state = 1;
    }
    c->t++;
  }
  return SCO_OK;
}

sco_status sco_observables(sco_ctx* c, sco_obs* o, int32_t want_full) {
  if (!c || !o) return SCO_EINVAL;
  const bool full = want_full && c->P.N <= 65536;
  if (c->graph_epoch >= 0 && !c->dip_valid) {
    SCO_TRY(dip_degree_run(c->P, c->row_ptr, c->col, c->cnt, c->st, &c->launches));
    c->dip_valid = true;
  }
  SCO_TRY(observables_run(c->P, c->s, c->row_ptr, c->col, c->tab.xy, c->graph_epoch >= 0, full,
                          c->cnt, c->st, &c->launches));
  sco_status st = read_counters(c);
  if (st != SCO_OK) return st;
  const DevCounters& h = *c->hcnt;
  const double N = (double)c->P.N;
  std::memset(o, 0, sizeof(*o));
  o->e_exchange = h.acc[4];
  o->e_switched = (c->graph_epoch >= 0 ? h.acc[5] : 0.0) + h.acc[4];
  o->e_full = full ? h.acc[6] : NAN;
  o->mx = h.acc[0] / N;
  o->my = h.acc[1] / N;
  o->mz = h.acc[2] / N;
  o->m_abs = std::sqrt(o->mx * o->mx + o->my * o->my + o->mz * o->mz);
  o->m_phi = h.acc[3] / N;
  const bool g = c->graph_epoch >= 0;
  o->n_edges = g ? (int64_t)h.n_dip : 0;
  o->max_degree = g ? (int32_t)h.max_degree : 0;
  o->max_degree_dipolar = g ? (int32_t)h.max_degree_dip : 0;
  o->n_colours = c->colour_valid ? (int32_t)h.n_colours : 0;
  o->kw_rounds = c->colour_valid ? (int32_t)h.kw_rounds : 0;
  o->sweeps_done = c->t;
  o->guard_hits_fp64 = (int64_t)h.guard_fp64;
  o->guard_hits_fp32 = (int64_t)h.guard_fp32;
  o->kernel_launches = c->launches;
  return SCO_OK;
}

sco_status sco_get_spins(sco_ctx* c, double* xyz, int32_t on_device) {
  if (!c || !xyz) return SCO_EINVAL;
  SCO_TRY(cudaMemcpyAsync(xyz, c->s, 3 * c->P.N * sizeof(double),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st));
  SCO_TRY(cudaStreamSynchronize(c->st));
  return c->sticky ? (sco_status)c->sticky : SCO_OK;
}

sco_status sco_set_spins(sco_ctx* c, const double* xyz, int32_t on_device) {
  if (!c || !xyz) return SCO_EINVAL;
  SCO_TRY(cudaMemcpyAsync(c->s, xyz, 3 * c->P.N * sizeof(double),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st));
  SCO_TRY(spins_to_f32(c->P.N, c->s, c->s32, c->st, &c->launches));
  SCO_TRY(cudaStreamSynchronize(c->st));
  c->cache_state = 2;  // the graph stays; its cached pair terms belong to the old spins
  return SCO_OK;
}

sco_status sco_get_sizes(sco_ctx* c, int64_t* n_sites, int64_t* n_entries, int32_t* max_degree,
                         int32_t* palette) {
  if (!c) return SCO_EINVAL;
  if (n_sites) *n_sites = c->P.N;
  if (n_entries) *n_entries = c->graph_epoch >= 0 ? (int64_t)c->nnz : 0;
  if (max_degree) *max_degree = c->graph_epoch >= 0 ? (int32_t)(c->g - 1) : 0;
  if (palette) *palette = c->graph_epoch >= 0 ? (int32_t)c->g : 0;
  return SCO_OK;
}

sco_status sco_get_graph(sco_ctx* c, uint32_t* row_ptr, uint32_t* col, uint32_t* colour) {
  if (!c) return SCO_EINVAL;
  if ((row_ptr || col) && c->graph_epoch < 0) return SCO_ESTATE;
  if (colour && !c->colour_valid) return SCO_ESTATE;
  if (row_ptr)
    SCO_TRY(cudaMemcpyAsync(row_ptr, c->row_ptr, (c->P.N + 1) * sizeof(uint32_t),
                            cudaMemcpyDeviceToHost, c->st));
  if (col && c->nnz) {
    // the device rows are unsorted: copy, sort every row by neighbour index, then read back
    uint32_t* tmp = nullptr;
    SCO_TRY(cudaMalloc(&tmp, c->nnz * sizeof(uint32_t)));
    cudaError_t e = csr_sorted_copy(c->P, c->row_ptr, c->col, tmp, c->nnz, c->cnt, c->st,
                                    &c->launches);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(col, tmp, c->nnz * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    cudaFree(tmp);
    SCO_TRY(e);
    c->dip_valid = true;
  }
  if (colour)
    SCO_TRY(cudaMemcpyAsync(colour, c->cb.colour, c->P.N * sizeof(uint32_t),
                            cudaMemcpyDeviceToHost, c->st));
  return read_counters(c);
}

sco_status sco_get_classes(sco_ctx* c, uint32_t* perm, uint32_t* off) {
  if (!c) return SCO_EINVAL;
  if (!c->colour_valid) return SCO_ESTATE;
  if (perm)
    SCO_TRY(cudaMemcpyAsync(perm, c->cb.perm, c->P.N * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                            c->st));
  if (off)
    SCO_TRY(cudaMemcpyAsync(off, c->cb.off, (c->g + 1) * sizeof(uint32_t),
                            cudaMemcpyDeviceToHost, c->st));
  return read_counters(c);
}

sco_status sco_get_accepts(sco_ctx* c, uint8_t* acc) {
  if (!c || !acc) return SCO_EINVAL;
  SCO_TRY(cudaMemcpyAsync(acc, c->acc, c->P.N, cudaMemcpyDeviceToHost, c->st));
  return read_counters(c);
}

sco_status sco_get_table(sco_ctx* c, int64_t* K, int32_t* dx, int32_t* dy, uint64_t* W,
                         double* cc) {
  if (!c) return SCO_EINVAL;
  const int64_t n = c->P.K;
  if (K) *K = n;
  if (n == 0) return SCO_OK;
  std::vector<uint32_t> d((size_t)n);
  SCO_TRY(cudaMemcpyAsync(d.data(), c->tab.disp, n * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                          c->st));
  if (W)
    SCO_TRY(cudaMemcpyAsync(W, c->tab.W, n * sizeof(uint64_t), cudaMemcpyDeviceToHost, c->st));
  std::vector<double2> xy;
  if (cc) {
    xy.resize((size_t)c->P.N);
    SCO_TRY(cudaMemcpyAsync(xy.data(), c->tab.xy, c->P.N * sizeof(double2),
                            cudaMemcpyDeviceToHost, c->st));
  }
  SCO_TRY(cudaStreamSynchronize(c->st));
  for (int64_t m = 0; m < n; ++m) {
    const int32_t x = (int16_t)(d[m] & 0xFFFFu), y = (int32_t)(d[m] >> 16);
    if (dx) dx[m] = x;
    if (dy) dy[m] = y;
    if (cc) {
      // the table holds fl(D c); report c itself only when D == 1 (tests), else D c
      cc[m] = xy[(size_t)((x < 0 ? -x : x) + (int64_t)c->P.Lx * y)].x;
    }
  }
  return SCO_OK;
}

sco_status sco_get_state(sco_ctx* c, void* buf, size_t* len) {
  if (!c || !len) return SCO_EINVAL;
  const int64_t N = c->P.N;
  const bool mid = c->p.n_sw > 1 && c->t % c->p.n_sw != 0 && c->graph_epoch == c->t / c->p.n_sw;
  const size_t need = sizeof(StateHeader) + (size_t)(mid ? 6 : 3) * N * sizeof(double);
  if (!buf) {
    *len = need;
    return SCO_OK;
  }
  if (*len < need) return SCO_EINVAL;
  StateHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "SCOSTAT1", 8);
  h.version = 1;
  h.has_epoch = mid ? 1 : 0;
  h.p = c->p;
  h.t = c->t;
  h.N = N;
  std::memcpy(buf, &h, sizeof(h));
  char* body = (char*)buf + sizeof(h);
  SCO_TRY(cudaMemcpyAsync(body, c->s, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  if (mid)
    SCO_TRY(cudaMemcpyAsync(body + 3 * N * sizeof(double), c->s_epoch, 3 * N * sizeof(double),
                            cudaMemcpyDeviceToHost, c->st));
  SCO_TRY(cudaStreamSynchronize(c->st));
  *len = need;
  return SCO_OK;
}

sco_status sco_set_state(sco_ctx* c, const void* buf, size_t len) {
  if (!c || !buf || len < sizeof(StateHeader)) return SCO_EINVAL;
  StateHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (std::memcmp(h.magic, "SCOSTAT1", 8) != 0 || h.version != 1) return SCO_ESTATE;
  const sco_params& a = h.p;
  const sco_params& b = c->p;
  if (a.Lx != b.Lx || a.Ly != b.Ly || a.J != b.J || a.D != b.D || a.T != b.T || a.seed != b.seed ||
      a.n_sw != b.n_sw || a.replica != b.replica || h.N != c->P.N || h.t < 0)
    return SCO_ESTATE;
  const int64_t N = c->P.N;
  const size_t need = sizeof(StateHeader) + (size_t)(h.has_epoch ? 6 : 3) * N * sizeof(double);
  if (len < need) return SCO_EINVAL;
  const char* body = (const char*)buf + sizeof(h);
  SCO_TRY(cudaMemcpyAsync(c->s, body, 3 * N * sizeof(double), cudaMemcpyHostToDevice, c->st));
  SCO_TRY(spins_to_f32(N, c->s, c->s32, c->st, &c->launches));
  c->t = h.t;
  c->graph_epoch = -1;
  c->colour_valid = false;
  if (h.has_epoch) {
    // rebuild the graph of the current epoch from the spins at its start
    if (!c->s_epoch) return SCO_ESTATE;
    SCO_TRY(cudaMemcpyAsync(c->s_epoch, body + 3 * N * sizeof(double), 3 * N * sizeof(double),
                            cudaMemcpyHostToDevice, c->st));
    float4* tmp32 = nullptr;
    SCO_TRY(cudaMalloc(&tmp32, N * sizeof(float4)));
    cudaError_t e = spins_to_f32(N, c->s_epoch, tmp32, c->st, &c->launches);
    sco_status st = e == cudaSuccess
                        ? do_switch(c, (uint32_t)(c->t / c->p.n_sw), c->s_epoch, tmp32)
                        : from_cuda(e);
    cudaStreamSynchronize(c->st);
    cudaFree(tmp32);
    if (st != SCO_OK) return st;
  }
  SCO_TRY(cudaStreamSynchronize(c->st));
  return SCO_OK;
}

sco_status sco_set_timing(sco_ctx* c, int32_t enable) {
  if (!c) return SCO_EINVAL;
  SCO_TRY(cudaStreamSynchronize(c->st));
  for (auto& e : c->evs) {
    c->pool.push_back(e.a);
    c->pool.push_back(e.b);
  }
  c->evs.clear();
  for (int k = 0; k < 3; ++k) {
    c->ms[k] = 0.0;
    c->calls[k] = 0;
  }
  c->timing = enable != 0;
  return SCO_OK;
}

sco_status sco_get_timing(sco_ctx* c, double ms[3], int64_t calls[3]) {
  if (!c) return SCO_EINVAL;
  SCO_TRY(cudaStreamSynchronize(c->st));
  for (auto& e : c->evs) {
    float t = 0.f;
    SCO_TRY(cudaEventElapsedTime(&t, e.a, e.b));
    c->ms[e.phase] += t;
    c->calls[e.phase] += 1;
    c->pool.push_back(e.a);
    c->pool.push_back(e.b);
  }
  c->evs.clear();
  for (int k = 0; k < 3; ++k) {
    if (ms) ms[k] = c->ms[k];
    if (calls) calls[k] = c->calls[k];
  }
  return SCO_OK;
}

sco_status sco_sync(sco_ctx* c) {
  if (!c) return SCO_EINVAL;
  return read_counters(c);
}

sco_status sco_set_temperature(sco_ctx* c, double T) {
  if (!c) return SCO_EINVAL;
  if (c->sticky) return (sco_status)c->sticky;
  sco_params q = c->p;
  q.T = T;
  if (!params_ok(&q)) return SCO_EINVAL;
  SCO_TRY(cudaStreamSynchronize(c->st));
  c->p = q;
  c->P = make_dev_params(q);
  // the temperature-dependent tables (pair energies scaled by beta, candidate probabilities)
  table_free_xy(c->tab);
  SCO_TRY(table_build_xy(c->P, c->tab, c->st, &c->launches));
  SCO_TRY(cudaStreamSynchronize(c->st));
  // the graph belongs to the old temperature: the next MC step switches again, same epoch
  c->graph_epoch = -1;
  c->colour_valid = false;
  return SCO_OK;
}

sco_status sco_get_graph_stats(sco_ctx* c, int32_t cells_x, int32_t cells_y, int32_t n_rbins,
                               sco_graph_stats* out, int64_t* survived, int64_t* pairs,
                               double* p_survive, double* delta_r) {
  if (!c || !out || cells_x < 1 || cells_y < 1 || cells_x > c->p.Lx || cells_y > c->p.Ly ||
      n_rbins < 1 || n_rbins > 4096)
    return SCO_EINVAL;
  if ((uint64_t)c->g * (uint64_t)cells_x * (uint64_t)cells_y > (1ull << 28)) return SCO_EINVAL;
  if (c->sticky) return (sco_status)c->sticky;
  if (c->graph_epoch < 0 || !c->colour_valid) return SCO_ESTATE;
  const size_t nb = (size_t)n_rbins;
  std::vector<unsigned long long> cnt(2 * nb + 1);
  std::vector<double> fo(6 + (size_t)c->g + nb);
  SCO_TRY(graph_stats_run(c->P, c->tab.disp, c->row_ptr, c->col, c->cb.colour, c->g, cells_x,
                          cells_y, n_rbins, c->st, &c->launches, cnt.data(), fo.data()));
  out->n_pairs = (int64_t)fo[0];
  out->n_cross = (int64_t)cnt[2 * nb];
  out->p_ipc = fo[2];
  out->delta_r_mean = fo[3];
  out->delta_r_max = fo[4];
  out->delta_r_weighted = fo[5];
  out->n_cells = cells_x * cells_y;
  out->palette = (int32_t)c->g;
  for (size_t b = 0; b < nb; ++b) {
    if (survived) survived[b] = (int64_t)cnt[b];
    if (pairs) pairs[b] = (int64_t)cnt[nb + b];
    if (p_survive) p_survive[b] = fo[6 + c->g + b];
  }
  if (delta_r)
    for (uint32_t k = 0; k < c->g; ++k) delta_r[k] = fo[6 + k];
  return read_counters(c);
}

sco_status sco_set_wait_limit(sco_ctx* c, uint64_t ns) {
  if (!c || ns > 3600000000000ull) return SCO_EINVAL;
  SCO_TRY(cudaStreamSynchronize(c->st));
  c->ns_limit = ns;
  return SCO_OK;
}

}  // extern "C"
