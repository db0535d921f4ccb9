// selftest.cu -- device self-test of the library's own elementary functions, expm1 (the degree-8
// expm1_np of the FP64 switch, the degree-6 expm1_np6 of the FP64 sweep decisions) on points of
// [-50, 0.35] and log_np (the FP64 candidate search of the switch) on points of (0, 1]: relative
// error against the double-double versions and difference from CUDA's.
#include <cstdint>
#include <cstring>

#include "sco.h"
#include "sco_internal.h"

namespace sco {
namespace {

__device__ __forceinline__ void atomic_max_pos(unsigned long long* a, double v) {
  atomicMax(a, (unsigned long long)__double_as_longlong(v));  // v >= 0: bits order like values
}

// Point k of n: fixed points (range ends, the -40 switch, reduction boundaries, tiny values),
// then n - 16 evenly spaced points of [-50, 0.35] each moved by a Philox fraction of the step.
template <int kDeg>
__global__ void k_expm1_test(int64_t n, uint64_t seed, dd ln2, unsigned long long* out) {
  const double fixed[16] = {-50.0,       -40.0,         -39.999999999, -0.34657359027997264,
                            -0.34657359027997270, -0.6931471805599453, -1.0397207708399179,
                            -1.0,        -1e-300,       -0x1p-30,      0.35,
                            0.0,         -20.0,         -2.0,          -0.5, 1e-10};
  double e_dd = 0.0, e_lib = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    double x;
    if (k < 16) {
      x = fixed[k];
    } else {
      const W4 w = philox((uint64_t)k, 0, 0, 7, seed, 0);
      x = -50.0 + 50.35 * ((double)(k - 16) + u53(w.w[0])) / (double)(n - 16);
    }
    if (x == 0.0) continue;
    const double y = expm1_np_deg<kDeg>(x);
    const dd r = dd_expm1(dd_from(x), ln2);
    const dd d = dd_sub(dd_from(y), r);
    e_dd = fmax(e_dd, fabs(d.hi / r.hi));
    const double yl = expm1(x);
    e_lib = fmax(e_lib, fabs((y - yl) / yl));
  }
  atomic_max_pos(&out[0], e_dd);
  atomic_max_pos(&out[1], e_lib);
}

// The library's log on n points of (0, 1] (16 fixed ones: 1 and its neighbours, the sqrt(2)/2
// switch, table boundaries, powers of two; then alternately 2^-e (1 + f) and 1 - 2^-e (1 + f) / 2
// with e in [1, 53] and f in [0, 1) from Philox: all octaves, and values just below 1), against
// the double-double log and CUDA's log.
__global__ void k_log_test(int64_t n, uint64_t seed, dd ln2, unsigned long long* out) {
  const double fixed[16] = {1.0, 0x1.fffffffffffffp-1, 0x1.ffffffffffffep-1, 0x1p-53,
                            0.5, 0x1.6a09e667f3bcdp-1, 0x1.6a09e667f3bccp-1, 0x1.6a09e667f3bcep-1,
                            0x1.ff8p-1, 0x1.ff7ffffffffffp-1, 0x1.008p0 * 0.5, 0.75,
                            0x1.0000000000001p-1, 0x1p-20, 0.999, 1e-10};
  double e_dd = 0.0, e_lib = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    double x;
    if (k < 16) {
      x = fixed[k];
    } else {
      const W4 w = philox((uint64_t)k, 0, 0, 9, seed, 0);
      const int e = 1 + (int)(w.w[0] % 53);
      const double f = u53(w.w[1]);
      x = (k & 1) ? 1.0 - ldexp(0.5 + 0.5 * f, -e) : ldexp(1.0 + f * (1.0 - 0x1p-53), -e);
    }
    const double y = log_np(x);
    if (x == 1.0) {
      e_dd = fmax(e_dd, fabs(y));  // exact 0 expected
      continue;
    }
    const dd r = dd_log(dd_from(x), ln2);
    const dd d = dd_sub(dd_from(y), r);
    e_dd = fmax(e_dd, fabs(d.hi / r.hi));
    const double yl = log(x);
    e_lib = fmax(e_lib, fabs((y - yl) / yl));
  }
  atomic_max_pos(&out[0], e_dd);
  atomic_max_pos(&out[1], e_lib);
}

dd ln2_dd() {  // ln 2 = 2 atanh(1/3) in double-double
  const dd third = dd_div(dd_from(1.0), dd_from(3.0));
  const dd x2 = dd_mul(third, third);
  dd pw = third, sum = dd_from(0.0);
  for (int k = 0; k < 40; ++k) {
    sum = dd_add(sum, dd_div(pw, dd_from(2.0 * k + 1.0)));
    pw = dd_mul(pw, x2);
  }
  return dd_ldexp(sum, 1);
}

// Runs test kernel `which` (0: expm1 degree 8, 1: expm1 degree 6, 2: log) on n points.
sco_status run_test(int which, int64_t n, uint64_t seed, double* err, double* diff) {
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return SCO_ECUDA;
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(unsigned long long)) != cudaSuccess) return SCO_ENOMEM;
  cudaError_t e = cudaMemset(d, 0, 2 * sizeof(unsigned long long));
  const dd ln2 = ln2_dd();
  if (e == cudaSuccess) {
    if (which == 0) k_expm1_test<8><<<1024, 256>>>(n, seed, ln2, d);
    else if (which == 1) k_expm1_test<6><<<1024, 256>>>(n, seed, ln2, d);
    else k_log_test<<<1024, 256>>>(n, seed, ln2, d);
    e = cudaGetLastError();
  }
  unsigned long long h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return SCO_ECUDA;
  double a, b;
  std::memcpy(&a, &h[0], 8);
  std::memcpy(&b, &h[1], 8);
  *err = a;
  if (diff) *diff = b;
  return SCO_OK;
}

// ---- FP64 throughput probe ------------------------------------------------------------
// Every thread advances kChains independent chains; a chain step is one FP64 FMA (kind 0),
// one expm1_np6 evaluation plus one FMA (kind 1, arguments kept in [-0.43, -0.3]) or one
// log_np evaluation plus one FMA (kind 2, arguments kept in [0.68, 0.75]).  The chains are
// independent, so with every warp slot of every SM filled the FP64 pipe, not the latency of
// one chain, bounds the rate.
constexpr int kProbeChains = 8;

template <int kKind>
__global__ void __launch_bounds__(256) k_probe_fp64(int64_t iters, double a, double b,
                                                    double* __restrict__ sink) {
  double x[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c)
    x[c] = (kKind == 2 ? 0.7 : -0.35) + 1e-6 * (double)((threadIdx.x + 37 * c) & 255);
  for (int64_t k = 0; k < iters; ++k) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) {
      if (kKind == 0) x[c] = fma(x[c], a, b);
      else if (kKind == 1) x[c] = fma(0.2, expm1_np_deg<6>(x[c]), -0.3);
      else x[c] = fma(0.1, log_np(x[c]), 0.75);
    }
  }
  double acc = 0.0;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) acc += x[c];
  if (acc == 1234.5) sink[0] = acc;  // never true: keeps the chains live
}

template <int kKind>
cudaError_t probe_one(int64_t iters, double* per_s) {
  int bps = 0, sms = 0, dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_probe_fp64<kKind>, 256, 0);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (bps < 1) bps = 1;
  const unsigned grid = (unsigned)(bps * sms);
  double* sink = nullptr;
  cudaEvent_t ea = nullptr, eb = nullptr;
  e = cudaMalloc(&sink, sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&ea);
  if (e == cudaSuccess) e = cudaEventCreate(&eb);
  if (e == cudaSuccess) {
    // warm-up launch (clocks, instruction cache), then the timed one
    k_probe_fp64<kKind><<<grid, 256>>>(iters / 8 + 1, 0.9999999, 1e-9, sink);
    e = cudaEventRecord(ea);
  }
  if (e == cudaSuccess) {
    k_probe_fp64<kKind><<<grid, 256>>>(iters, 0.9999999, 1e-9, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(eb);
  if (e == cudaSuccess) e = cudaEventSynchronize(eb);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ea, eb);
  if (e == cudaSuccess)
    *per_s = (double)grid * 256.0 * (double)iters * kProbeChains / (ms * 1e-3);
  if (ea) cudaEventDestroy(ea);
  if (eb) cudaEventDestroy(eb);
  cudaFree(sink);
  return e;
}

}  // namespace
}  // namespace sco

using namespace sco;

extern "C" sco_status sco_probe_fp64(int64_t iters, double out[3]) {
  if (iters < 1 || iters > (1ll << 30) || !out) return SCO_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return SCO_ECUDA;
  if (probe_one<0>(iters, &out[0]) != cudaSuccess) return SCO_ECUDA;
  // the elementary functions cost about a dozen FMAs each: fewer steps for the same time
  const int64_t it2 = iters / 12 > 0 ? iters / 12 : 1;
  if (probe_one<1>(it2, &out[1]) != cudaSuccess) return SCO_ECUDA;
  if (probe_one<2>(it2, &out[2]) != cudaSuccess) return SCO_ECUDA;
  return SCO_OK;
}

extern "C" sco_status sco_selftest_expm1_deg(int64_t n, uint64_t seed, int32_t degree,
                                             double* max_rel_err, double* max_rel_diff_cuda) {
  if (n < 17 || !max_rel_err || (degree != 6 && degree != 8)) return SCO_EINVAL;
  return run_test(degree == 8 ? 0 : 1, n, seed, max_rel_err, max_rel_diff_cuda);
}

extern "C" sco_status sco_selftest_log(int64_t n, uint64_t seed, double* max_rel_err,
                                       double* max_rel_diff_cuda) {
  if (n < 17 || !max_rel_err) return SCO_EINVAL;
  return run_test(2, n, seed, max_rel_err, max_rel_diff_cuda);
}

extern "C" sco_status sco_selftest_expm1(int64_t n, uint64_t seed, double* max_rel_err,
                                         double* max_rel_diff_cuda) {
  return sco_selftest_expm1_deg(n, seed, 8, max_rel_err, max_rel_diff_cuda);
}
