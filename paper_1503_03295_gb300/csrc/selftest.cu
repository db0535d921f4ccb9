// selftest.cu -- device self-test of the library's own elementary function expm1 (the degree-8
// expm1_np of the FP64 switch, the degree-6 expm1_np6 of the FP64 sweep decisions): its relative
// error against the double-double expm1 and its difference from the CUDA expm1, on points
// spread over [-50, 0.35].
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

}  // namespace
}  // namespace sco

using namespace sco;

extern "C" sco_status sco_selftest_expm1_deg(int64_t n, uint64_t seed, int32_t degree,
                                             double* max_rel_err, double* max_rel_diff_cuda) {
  if (n < 17 || !max_rel_err || (degree != 6 && degree != 8)) return SCO_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return SCO_ECUDA;
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(unsigned long long)) != cudaSuccess) return SCO_ENOMEM;
  cudaError_t e = cudaMemset(d, 0, 2 * sizeof(unsigned long long));
  // ln 2 = 2 atanh(1/3) in double-double
  const dd third = dd_div(dd_from(1.0), dd_from(3.0));
  const dd x2 = dd_mul(third, third);
  dd pw = third, sum = dd_from(0.0);
  for (int k = 0; k < 40; ++k) {
    sum = dd_add(sum, dd_div(pw, dd_from(2.0 * k + 1.0)));
    pw = dd_mul(pw, x2);
  }
  const dd ln2 = dd_ldexp(sum, 1);
  if (e == cudaSuccess) {
    if (degree == 8) k_expm1_test<8><<<1024, 256>>>(n, seed, ln2, d);
    else k_expm1_test<6><<<1024, 256>>>(n, seed, ln2, d);
    e = cudaGetLastError();
  }
  unsigned long long h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return SCO_ECUDA;
  double a, b;
  std::memcpy(&a, &h[0], 8);
  std::memcpy(&b, &h[1], 8);
  *max_rel_err = a;
  if (max_rel_diff_cuda) *max_rel_diff_cuda = b;
  return SCO_OK;
}

extern "C" sco_status sco_selftest_expm1(int64_t n, uint64_t seed, double* max_rel_err,
                                         double* max_rel_diff_cuda) {
  return sco_selftest_expm1_deg(n, seed, 8, max_rel_err, max_rel_diff_cuda);
}
