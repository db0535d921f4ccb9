// table.cu -- the translation-invariant coupling table, built on the device.
//
// Every unordered pair of the open lattice is (i, i + d) for one d of the half plane
// {dy > 0, |dx| < Lx} u {dy = 0, 0 < dx < Lx}.  The list is sorted by (r^2, dy, dx) with a
// stable counting sort on r^2 (rows are placed in increasing dy, and inside a row the
// negative dx before the positive one), each element carries the integer hazard
// A(r^2) > 2^60 / r^3 of its pair (V_max = D A 2^-59 >= 2D / r^3, Sec. 2.1), and W is the
// inclusive prefix of A.  A second table indexed by (|dx|, |dy|) holds fl(D c(r^2)) and
// V_max for the pair-energy evaluations of the switch and sweep kernels.
#include <cstdint>

#include "sco_internal.h"

namespace sco {

namespace {

__device__ __forceinline__ void disp_of_q(int64_t q, int32_t Lx, int32_t& dx, int32_t& dy) {
  if (q < Lx - 1) {
    dx = (int32_t)q + 1;
    dy = 0;
    return;
  }
  const int64_t r = q - (Lx - 1);
  const int64_t w = 2 * (int64_t)Lx - 1;
  dy = (int32_t)(r / w) + 1;
  dx = (int32_t)(r % w) - (Lx - 1);
}

__global__ void k_r2_count(int32_t Lx, int64_t K, uint32_t* __restrict__ cnt) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= K) return;
  int32_t dx, dy;
  disp_of_q(q, Lx, dx, dy);
  atomicAdd(&cnt[(int64_t)dx * dx + (int64_t)dy * dy], 1u);
}

// One block walks the rows dy = 0..Ly-1 in order.  Inside a row the values |dx| are
// distinct, hence so are the r^2, so the threads of a row never touch the same bucket.
__global__ void __launch_bounds__(1024) k_order(int32_t Lx, int32_t Ly,
                                                const uint32_t* __restrict__ start,
                                                uint32_t* __restrict__ seen,
                                                uint32_t* __restrict__ disp) {
  for (int32_t dy = 0; dy < Ly; ++dy) {
    for (int32_t ax = threadIdx.x; ax < Lx; ax += blockDim.x) {
      if (dy == 0 && ax == 0) continue;
      const int64_t r2 = (int64_t)ax * ax + (int64_t)dy * dy;
      uint32_t m = start[r2] + seen[r2];
      uint32_t n = 0;
      if (dy > 0 && ax > 0) {  // (-ax, dy) precedes (ax, dy)
        disp[m++] = ((uint32_t)(uint16_t)(int16_t)(-ax)) | ((uint32_t)dy << 16);
        ++n;
      }
      disp[m] = ((uint32_t)(uint16_t)(int16_t)ax) | ((uint32_t)dy << 16);
      ++n;
      seen[r2] += n;
    }
    __syncthreads();
  }
}

__global__ void k_hazard(int64_t K, const uint32_t* __restrict__ disp, uint64_t* __restrict__ A) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= K) return;
  const uint32_t d = disp[m];
  const int32_t dx = (int16_t)(d & 0xFFFFu), dy = (int32_t)(d >> 16);
  A[m] = hazard_A((int64_t)dx * dx + (int64_t)dy * dy);
}

// Sweep constants of a pair at (|dx|, |dy|).  FP64 (Sw64): the field of S_j on site i scaled
// by beta, f = a1 S_j - (S_j . a3 d) d with a1 = fl(beta fl(Dc r^2)) and a3 d = fl(beta fl(3 Dc)) d,
// so x = beta V - fl(beta Vmax) = S_i . f - bvm; c0 bounds the part of |x error| that does not
// scale with |x|: |beta dV| <= 2^-46 beta Dc r^2 (FP64 products, the rounded beta-scaled
// constants) plus 2^-51 beta Vmax (fl(beta Vmax)), plus 2^-52 (2 beta Vmax) for the rounding of
// x itself (|x| <= 2 beta Vmax).  The switch's survival test uses the same x.  FP32 (float4 {A1, A3, beta Vmax, c0}): V(S) = S.f with
// f = A1 S_j - A3 (S_j.d) d, |dV| <= 2^-16 Dc r^2 (shadow spins, FP32 constants).
__global__ void k_xy(int32_t Lx, int32_t Ly, double D, double beta, double2* __restrict__ xy,
                     double* __restrict__ xyq, float4* __restrict__ xy32,
                     Sw64* __restrict__ sw64, float4* __restrict__ sw32) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= (int64_t)Lx * Ly) return;
  const int64_t ax = q % Lx, ay = q / Lx;
  const int64_t r2 = ax * ax + ay * ay;
  double dc = 0.0, vm = 0.0;
  if (r2 > 0) {
    dc = __dmul_rn(D, coupling_c(r2));
    vm = __dmul_rn(__dmul_rn(D, (double)hazard_A(r2)), 0x1p-59);
  }
  const double a = (2.0 * beta) * vm;
  const double cq = -expm1(-a);
  xy[q] = make_double2(dc, vm);
  xyq[q] = cq;
  xy32[q] = make_float4((float)dc, (float)vm, (float)a, (float)cq);
  const double a1 = dc * (double)r2, a3 = 3.0 * dc, bvm = beta * vm;
  const double a3b = beta * a3;
  const double c64 = beta * (0x1p-46 * dc * (double)r2) + 0x1p-51 * bvm + 0x1p-52 * (2.0 * bvm);
  Sw64 t;
  t.a1 = beta * a1;
  t.a3x = a3b * (double)ax;
  t.a3y = a3b * (double)ay;
  t.ax = (double)ax;
  t.ay = (double)ay;
  t.bvm = bvm;
  t.c0 = c64 * (1.0 + 0x1p-20);
  // survival test of the switch: mu = (1 - P) - u q with 1 - P = -expm1_np6(x): |d(1 - P)| <=
  // |dx| <= c0 plus the relative error of expm1_np6 (bounded at run time, see survives_fp64); q
  // (CUDA expm1 of a rounded 2 beta Vmax) within 2^-50; the product u q and the difference 2^-52
  // each.  Doubled, and doubled again for the test against the larger of the two parts.
  t.bsw = 4.0 * (c64 + 0x1p-49) * (1.0 + 0x1p-20);
  sw64[q] = t;
  const double c32 = beta * (0x1p-16 * dc * (double)r2) + 0x1p-21 * bvm;
  sw32[q] = make_float4((float)a1, (float)a3, (float)bvm, (float)(c32 * (1.0 + 0x1p-20)));
}

// exp(x) of a double-double x <= 0 without the cancellation of 1 + expm1(x): x = k ln2 + r,
// |r| <= ln2 / 2, e^x = 2^k (1 + expm1(r)); relative error of the double-double result far below
// 2^-100 (the series and the reduction of dd_expm1_small / dd_expm1).
__device__ dd exp_dd_neg(dd x, dd ln2) {
  const double kf = floor(x.hi / ln2.hi + 0.5);
  const dd r = dd_sub(x, dd_mul_d(ln2, kf));
  return dd_ldexp(dd_add(dd_from(1.0), dd_expm1_small(r)), (int)kf);
}

// E_m = fl(exp(-beta D 2^-58 W_m)) as bits: the candidate process of the switch has rate
// beta D A_m 2^-58 per element, so E_m is the probability of passing elements 0..m without a
// candidate.  The exponent is formed exactly (beta D as a double-double product, W_m split into
// two exact doubles), the exponential in double-double and rounded once, so E_m lies within
// 2^-52 of its exact value (relative); below e^-690 (< 2^-995) it is stored as +0, which the
// search treats as below every target it accepts (targets under 2^-990 take the exact path).
__global__ void k_decay(int64_t K, double beta, double D, double ln2_hi, double ln2_lo,
                        const uint64_t* __restrict__ W, uint64_t* __restrict__ Eb) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= K) return;
  const uint64_t w = W[m];
  const dd wd = dd_add(dd_from((double)(w >> 32) * 0x1p32), dd_from((double)(w & 0xFFFFFFFFull)));
  const dd a = dd_ldexp(dd_mul(two_prod(beta, D), wd), -58);
  double e = 0.0;
  if (a.hi < 690.0) {
    const dd x = exp_dd_neg(dd_neg(a), dd{ln2_hi, ln2_lo});
    e = x.hi + x.lo;
  }
  Eb[m] = (uint64_t)__double_as_longlong(e);
}

}  // namespace

cudaError_t table_build_xy(const DevParams& P, Table& t, cudaStream_t s, int64_t* launches) {
  cudaError_t e;
  const int64_t nxy = (int64_t)P.Lx * P.Ly;
  if ((e = cudaMalloc(&t.xy, nxy * sizeof(double2))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&t.xy32, nxy * sizeof(float4))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&t.xyq, nxy * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&t.sw64, nxy * sizeof(Sw64))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&t.sw32, nxy * sizeof(float4))) != cudaSuccess) return e;
  k_xy<<<(unsigned)((nxy + 255) / 256), 256, 0, s>>>(P.Lx, P.Ly, P.D, P.beta, t.xy, t.xyq,
                                                      t.xy32, t.sw64, t.sw32);
  ++*launches;
  // the FP64 candidate search's decay values, where this table owns the sorted list
  if (t.W && t.K > 0) {
    if ((e = cudaMalloc(&t.Ebits, t.K * sizeof(uint64_t))) != cudaSuccess) return e;
    k_decay<<<(unsigned)((t.K + 255) / 256), 256, 0, s>>>(t.K, P.beta, P.D, P.ln2_hi, P.ln2_lo,
                                                          t.W, t.Ebits);
    ++*launches;
  }
  return cudaGetLastError();
}

cudaError_t table_build_list(const DevParams& P, Table& t, cudaStream_t s, int64_t* launches) {
  cudaError_t e;
  const int64_t K = P.K;
  t.K = K;
  if ((e = cudaMalloc(&t.disp, (K > 0 ? K : 1) * sizeof(uint32_t))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&t.W, (K > 0 ? K : 1) * sizeof(uint64_t))) != cudaSuccess) return e;
  if (K == 0) return cudaGetLastError();
  const int64_t R2 = (int64_t)(P.Lx - 1) * (P.Lx - 1) + (int64_t)(P.Ly - 1) * (P.Ly - 1);
  uint32_t *cnt = nullptr, *start = nullptr;
  uint64_t *A = nullptr, *tmp = nullptr;
  const int64_t ns = (R2 + 2 > K ? R2 + 2 : K);
  e = cudaMalloc(&cnt, (R2 + 2) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&start, (R2 + 2) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&A, K * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&tmp, scan_tmp_bytes(ns));
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, (R2 + 2) * sizeof(uint32_t), s);
  if (e == cudaSuccess) {
    k_r2_count<<<(unsigned)((K + 255) / 256), 256, 0, s>>>(P.Lx, K, cnt);
    ++*launches;
    e = scan_excl_u32(cnt, start, R2 + 1, tmp, nullptr, s, launches);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, (R2 + 2) * sizeof(uint32_t), s);
  if (e == cudaSuccess) {
    k_order<<<1, 1024, 0, s>>>(P.Lx, P.Ly, start, cnt, t.disp);
    ++*launches;
    k_hazard<<<(unsigned)((K + 255) / 256), 256, 0, s>>>(K, t.disp, A);
    ++*launches;
    e = scan_incl_u64(A, t.W, K, tmp, nullptr, s, launches);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(cnt);
  cudaFree(start);
  cudaFree(A);
  cudaFree(tmp);
  if (e != cudaSuccess) return e;
  // table index of the two nearest-neighbour displacements (1,0) and (0,1)
  uint32_t head[2] = {0, 0};
  const int nh = K < 2 ? (int)K : 2;
  if ((e = cudaMemcpy(head, t.disp, nh * sizeof(uint32_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return e;
  for (int q = 0; q < nh; ++q) {
    if (head[q] == 1u) t.m_nn[0] = q;
    if (head[q] == (1u << 16)) t.m_nn[1] = q;
  }
  return cudaGetLastError();
}

cudaError_t table_build(const DevParams& P, Table& t, cudaStream_t s, int64_t* launches) {
  cudaError_t e = table_build_list(P, t, s, launches);
  if (e == cudaSuccess) e = table_build_xy(P, t, s, launches);
  return e;
}

void table_free_xy(Table& t) {
  cudaFree(t.xy);
  cudaFree(t.xy32);
  cudaFree(t.xyq);
  cudaFree(t.sw64);
  cudaFree(t.sw32);
  cudaFree(t.Ebits);
  t.Ebits = nullptr;
  t.xy = nullptr;
  t.xy32 = nullptr;
  t.xyq = nullptr;
  t.sw64 = nullptr;
  t.sw32 = nullptr;
}

void table_free(Table& t) {
  cudaFree(t.disp);
  cudaFree(t.W);
  table_free_xy(t);
  t = Table();
}

}  // namespace sco
