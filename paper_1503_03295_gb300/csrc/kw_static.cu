// kw_static.cu -- Kuhn-Wattenhofer colouring of a caller's CSR graph that allocates nothing.
//
// Same colouring as sco_colour (one barrier-free dataflow kernel per level, see colour.cu),
// for callers that cannot let a library allocate device memory.  Its working memory is one
// file-scope device array of fixed size: per-vertex words for up to
// SCO_KW_STATIC_MAX_VERTICES vertices followed by a small control block.  Every call
// shares that array; calls that overlap on the GPU race.
#include <cstdint>
#include <cstring>
#include <mutex>

#include "sco.h"
#include "sco_internal.h"

namespace {

using namespace sco;

constexpr int64_t kMaxVertices = SCO_KW_STATIC_MAX_VERTICES;
constexpr int kCtrlWords = 64;  // 512 bytes of control block after the vertex words
constexpr int kMaxDevices = 64;
constexpr int kStatusTimeout = 4;
constexpr unsigned long long kColMask = 0xFFFFFFFFull;

struct StaticCtrl {
  unsigned int max_degree;
  unsigned int g;
  unsigned int levels;
  int status;
  unsigned long long magic;  // multiplier of g (div_magic)
  unsigned int kw_rounds;
  unsigned int pad;
  unsigned int lev_rounds[32];
};
static_assert(sizeof(StaticCtrl) <= kCtrlWords * 8, "control block");

// The scratch: kMaxVertices packed words, then the control block.  8 MiB + 512 B per device.
static __device__ __align__(256) unsigned long long g_kw_scratch[kMaxVertices + kCtrlWords];

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
__device__ __forceinline__ int ld_status(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t fdiv(uint32_t u, unsigned long long M) {
  return div_by_magic(u, M);  // M = 0 stands for g = 1
}

__global__ void k_st_degree(uint32_t n, const uint32_t* __restrict__ row_ptr,
                            StaticCtrl* __restrict__ ctrl) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned d = v < n ? row_ptr[v + 1] - row_ptr[v] : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d = max(d, __shfl_down_sync(0xffffffffu, d, o));
  if ((threadIdx.x & 31) == 0 && d) atomicMax(&ctrl->max_degree, d);
}

__global__ void k_st_setup(uint32_t n, StaticCtrl* __restrict__ ctrl) {
  const unsigned g = ctrl->max_degree + 1;
  const uint32_t G = (n + g - 1) / g;
  unsigned M = 0;
  while ((1u << M) < G) ++M;
  ctrl->g = g;
  ctrl->levels = M;
  ctrl->magic = div_magic(g);
}

__global__ void k_st_init(uint32_t n, unsigned long long* __restrict__ word,
                          const StaticCtrl* __restrict__ ctrl) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) word[v] = pack(0, 0, v % ctrl->g);
}

__device__ __noinline__ unsigned st_mex_slow(uint32_t v, unsigned p, unsigned long long M,
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

// One KW level (modified reduction (2)'); g, M and the divisor constant come from the
// control block, and levels beyond M return at once.
__global__ void __launch_bounds__(256) k_st_level(uint32_t n, unsigned p,
                                                  const uint32_t* __restrict__ row_ptr,
                                                  const uint32_t* __restrict__ col,
                                                  unsigned long long* word,
                                                  StaticCtrl* __restrict__ ctrl,
                                                  unsigned long long ns_limit) {
  if (p > ctrl->levels) return;
  const unsigned long long t_start = global_ns();
  const uint32_t g = ctrl->g;
  const unsigned long long M = ctrl->magic;
  const uint32_t half = g << (p - 1);
  const uint32_t ngroups = (uint32_t)(((unsigned long long)n + ((unsigned long long)g << p) - 1) /
                                      ((unsigned long long)g << p));
  const uint32_t R = ngroups * half;
  const uint32_t nth = gridDim.x * blockDim.x;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned rmax = 0;
  unsigned nap = 64;  // back-off (ns) after a pass in which none of this thread's vertices moved
  bool pending = true;
  for (unsigned long long pass = 0; pending; ++pass) {
    pending = false;
    bool progress = false;
    for (uint32_t r = tid; r < R; r += nth) {
      const uint32_t k = fdiv(r, M) >> (p - 1);
      const uint32_t v = (2 * k + 1) * half + (r - k * half);
      if (v >= n) continue;
      const unsigned long long wv = ld_relaxed(&word[v]);
      if (tag_of(wv) == p) continue;
      const uint32_t cv = (uint32_t)(wv & kColMask);
      const uint32_t b = row_ptr[v], e = row_ptr[v + 1];
      unsigned long long used[4] = {0, 0, 0, 0};
      bool blocked = false;
      unsigned rv = 0;
      for (uint32_t q = b; q < e; ++q) {
        const uint32_t u = col[q] & kIndexMask;
        const uint32_t gu = fdiv(u, M);
        if ((gu >> p) != k) continue;
        const unsigned long long wu = ld_relaxed(&word[u]);
        const uint32_t cu = (uint32_t)(wu & kColMask);
        const bool right = (gu >> (p - 1)) & 1u;
        if (right && tag_of(wu) != p) {
          if (cu > cv) {
            blocked = true;
            break;
          }
          continue;
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
        c = st_mex_slow(v, p, M, row_ptr, col, word);
      }
      rmax = max(rmax, rv + 1);
      st_relaxed(&word[v], pack(p, rv + 1, c));
      progress = true;
    }
    if (pending) {
      if (progress) {
        nap = 64;
      } else {
        __nanosleep(nap);
        nap = nap < 2048 ? 2 * nap : 2048;
      }
    }
    if (pending && ((pass & 15) == 15) &&
        (global_ns() - t_start > ns_limit || ld_status(&ctrl->status) != 0)) {
      atomicCAS(&ctrl->status, 0, kStatusTimeout);
      break;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rmax = max(rmax, __shfl_down_sync(0xffffffffu, rmax, o));
  if ((threadIdx.x & 31) == 0 && rmax) atomicMax(&ctrl->lev_rounds[p & 31], rmax);
}

__global__ void k_st_final(uint32_t n, int variant, const unsigned long long* __restrict__ word,
                           uint32_t* __restrict__ colour, StaticCtrl* __restrict__ ctrl) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) colour[v] = (uint32_t)(word[v] & kColMask);
  if (v == 0) {
    unsigned t = 0;
    for (unsigned p = 1; p <= ctrl->levels; ++p) t += ctrl->lev_rounds[p & 31];
    ctrl->kw_rounds = variant == 1 ? ctrl->g * ctrl->levels : t;
  }
}

std::mutex g_setup_mu;
unsigned long long* g_scratch_addr[kMaxDevices] = {};
int g_blocks_per_sm[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

}  // namespace

extern "C" sco_status sco_kw_colour_static(const uint32_t* row_ptr, const uint32_t* col,
                                           int64_t n, int32_t variant, uint32_t* colour,
                                           int32_t* max_degree, int32_t* rounds, void* stream) {
  if (n < 0 || n > kMaxVertices || variant < 0 || variant > 1) return SCO_EINVAL;
  if (n == 0) {
    if (max_degree) *max_degree = 0;
    if (rounds) *rounds = 0;
    return SCO_OK;
  }
  if (!row_ptr || !col || !colour) return SCO_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SCO_ECUDA;
  unsigned long long* base = nullptr;
  {
    // once per device, with that device current: the device address of the scratch array
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_kw_scratch) != cudaSuccess || !p) return SCO_ECUDA;
      int bps = 0, sms = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_st_level, 256, 0) != cudaSuccess)
        return SCO_ECUDA;
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SCO_ECUDA;
      g_blocks_per_sm[dev] = bps > 0 ? bps : 1;
      g_sms[dev] = sms > 0 ? sms : 1;
      g_scratch_addr[dev] = (unsigned long long*)p;
    }
    base = g_scratch_addr[dev];
  }
  unsigned long long* word = base;
  StaticCtrl* ctrl = reinterpret_cast<StaticCtrl*>(base + kMaxVertices);
  const uint32_t nn = (uint32_t)n;
  if (cudaMemsetAsync(ctrl, 0, sizeof(StaticCtrl), st) != cudaSuccess) return SCO_ECUDA;
  const unsigned nb = (nn + 255) / 256;
  k_st_degree<<<nb, 256, 0, st>>>(nn, row_ptr, ctrl);
  k_st_setup<<<1, 1, 0, st>>>(nn, ctrl);
  k_st_init<<<nb, 256, 0, st>>>(nn, word, ctrl);
  if (cudaGetLastError() != cudaSuccess) return SCO_ECUDA;
  unsigned pmax = 0;  // g >= 1 bounds the level count by ceil(log2 n)
  while ((1ull << pmax) < (unsigned long long)n) ++pmax;
  int64_t grid = (int64_t)g_blocks_per_sm[dev] * g_sms[dev];
  const int64_t want = ((int64_t)nn / 2 + 255) / 256;
  if (want < grid) grid = want > 0 ? want : 1;
  unsigned long long ns_limit = 2000000000ull;
  for (unsigned p = 1; p <= pmax; ++p) {
    uint32_t a0 = nn;
    unsigned a1 = p;
    void* args[] = {(void*)&a0, (void*)&a1, (void*)&row_ptr, (void*)&col, (void*)&word,
                    (void*)&ctrl, (void*)&ns_limit};
    if (cudaLaunchCooperativeKernel((const void*)k_st_level, dim3((unsigned)grid), dim3(256), args,
                                    0, st) != cudaSuccess)
      return SCO_ECUDA;
  }
  k_st_final<<<nb, 256, 0, st>>>(nn, variant, word, colour, ctrl);
  StaticCtrl h;
  std::memset(&h, 0, sizeof(h));
  if (cudaMemcpyAsync(&h, ctrl, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return SCO_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SCO_ECUDA;
  if (h.status != 0) return (sco_status)h.status;
  if (max_degree) *max_degree = (int32_t)h.max_degree;
  if (rounds) *rounds = (int32_t)h.kw_rounds;
  return SCO_OK;
}
