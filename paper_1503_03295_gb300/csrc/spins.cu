// spins.cu -- initial spins and the observables of the SCO chain.
#include <cmath>
#include <cstdint>

#include "sco_internal.h"

namespace sco {

namespace {

// Uniform initial spins: Philox tag INIT, counter (i, 0, a), Marsaglia attempt a = 0..63;
// (0, 0, 1) if all 64 attempts fail (probability ~1e-43).
__global__ void k_init(DevParams P, double* __restrict__ s, float4* __restrict__ s32) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= P.N) return;
  double x = 0.0, y = 0.0, z = 1.0;
  for (uint64_t a = 0; a < 64; ++a) {
    const W4 w = philox((uint64_t)i, 0, a, kTagInit, P.key0, P.key1);
    if (marsaglia(w.w[0], w.w[1], x, y, z)) break;
    x = 0.0; y = 0.0; z = 1.0;
  }
  s[i] = x;
  s[P.N + i] = y;
  s[2 * P.N + i] = z;
  if (s32) s32[i] = make_float4((float)x, (float)y, (float)z, 0.f);
}

__global__ void k_to_f32(int64_t n, const double* __restrict__ s, float4* __restrict__ s32) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) s32[i] = make_float4((float)s[i], (float)s[n + i], (float)s[2 * n + i], 0.f);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sums of up to 8 accumulators, then one atomicAdd per block and accumulator.
template <int NA>
__device__ __forceinline__ void block_accumulate(double (&v)[NA], double* dst) {
  __shared__ double red[NA][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    const double w = warp_sum(v[a]);
    if (lane == 0) red[a][wid] = w;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      double w = lane < nw ? red[a][lane] : 0.0;
      w = warp_sum(w);
      if (lane == 0) atomicAdd(&dst[a], w);
    }
  }
}

// Site sums: magnetisation, the circular component of Eq. (7) and the exchange energy
// -J sum_<ij> S_i.S_j.  acc[0..2] = sum S, acc[3] = sum [S x u^]_z, acc[4] = exchange.
__global__ void __launch_bounds__(256) k_site_obs(DevParams P, const double* __restrict__ s,
                                                  double* __restrict__ acc) {
  double v[5] = {0, 0, 0, 0, 0};
  const double rcx = 0.5 * (P.Lx - 1), rcy = 0.5 * (P.Ly - 1);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = s[i], y = s[P.N + i], z = s[2 * P.N + i];
    v[0] += x;
    v[1] += y;
    v[2] += z;
    const int32_t yi = (int32_t)site_row((uint32_t)i, P);
    const int32_t xi = (int32_t)((uint32_t)i - (uint32_t)yi * (uint32_t)P.Lx);
    const double ux = xi - rcx, uy = yi - rcy;
    const double nr = sqrt(ux * ux + uy * uy);
    if (nr > 0.0) v[3] += (x * uy - y * ux) / nr;
    if (P.J != 0.0) {
      if (xi + 1 < P.Lx)
        v[4] += x * s[i + 1] + y * s[P.N + i + 1] + z * s[2 * P.N + i + 1];
      if (yi + 1 < P.Ly) {
        const int64_t j = i + P.Lx;
        v[4] += x * s[j] + y * s[P.N + j] + z * s[2 * P.N + j];
      }
    }
  }
  v[4] *= -P.J;
  block_accumulate<5>(v, acc);
}

// Pseudointeraction energy H' of Eq. (4) over surviving dipolar pairs (each once, i < j):
// Vbar = V - beta^-1 log(1 - exp(beta (V - Vmax))).  acc[5].
__global__ void __launch_bounds__(256) k_pair_obs(DevParams P, const double* __restrict__ s,
                                                  const uint32_t* __restrict__ row_ptr,
                                                  const uint32_t* __restrict__ col,
                                                  const double2* __restrict__ xy,
                                                  double* __restrict__ acc) {
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t yi = (int32_t)site_row((uint32_t)i, P);
    const int32_t xi = (int32_t)((uint32_t)i - (uint32_t)yi * (uint32_t)P.Lx);
    const double ax = s[i], ay = s[P.N + i], az = s[2 * P.N + i];
    for (uint32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      const uint32_t c = col[e];
      if (c & kExchOnly) continue;
      const int64_t j = c;
      if (j <= i) continue;
      const uint32_t yj = site_row((uint32_t)j, P);
      const int32_t dx = (int32_t)((uint32_t)j - yj * (uint32_t)P.Lx) - xi, dy = (int32_t)yj - yi;
      const double2 t = xy[(int64_t)(dx < 0 ? -dx : dx) + (int64_t)P.Lx * (dy < 0 ? -dy : dy)];
      const double V = pair_V(t.x, (double)dx * dx + (double)dy * dy, ax, ay, az, s[j],
                              s[P.N + j], s[2 * P.N + j], (double)dx, (double)dy);
      const double xx = P.beta * (V - t.y);
      const double l = xx > -0.6931471805599453 ? log(-expm1(xx)) : log1p(-exp(xx));
      v[0] += V - l / P.beta;
    }
  }
  block_accumulate<1>(v, acc + 5);
}

// Full H of Eq. (6) by direct summation over all pairs (tiles of 256 j per block row).
__global__ void __launch_bounds__(256) k_full_energy(DevParams P, const double* __restrict__ s,
                                                     double* __restrict__ acc) {
  __shared__ double sj[3][256];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool ok = i < P.N;
  const double ax = ok ? s[i] : 0, ay = ok ? s[P.N + i] : 0, az = ok ? s[2 * P.N + i] : 0;
  const int32_t xi = ok ? (int32_t)(i % P.Lx) : 0, yi = ok ? (int32_t)(i / P.Lx) : 0;
  double e = 0.0;
  for (int64_t j0 = 0; j0 < P.N; j0 += 256) {
    const int64_t jl = j0 + threadIdx.x;
    sj[0][threadIdx.x] = jl < P.N ? s[jl] : 0;
    sj[1][threadIdx.x] = jl < P.N ? s[P.N + jl] : 0;
    sj[2][threadIdx.x] = jl < P.N ? s[2 * P.N + jl] : 0;
    __syncthreads();
    const int64_t jn = (P.N - j0 < 256) ? P.N - j0 : 256;
    if (ok) {
      for (int k = 0; k < jn; ++k) {
        const int64_t j = j0 + k;
        if (j <= i) continue;
        const int32_t dx = (int32_t)(j % P.Lx) - xi, dy = (int32_t)(j / P.Lx) - yi;
        const double r2 = (double)dx * dx + (double)dy * dy;
        const double bx = sj[0][k], by = sj[1][k], bz = sj[2][k];
        const double c = 1.0 / (r2 * r2 * sqrt(r2));
        e += pair_V(P.D * c, r2, ax, ay, az, bx, by, bz, (double)dx, (double)dy);
        if (r2 == 1.0) e -= P.J * (ax * bx + ay * by + az * bz);
      }
    }
    __syncthreads();
  }
  double v[1] = {e};
  block_accumulate<1>(v, acc + 6);
}

}  // namespace

cudaError_t spins_init(const DevParams& P, double* s, float4* s32, cudaStream_t st,
                       int64_t* launches) {
  k_init<<<(unsigned)((P.N + 255) / 256), 256, 0, st>>>(P, s, s32);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t spins_to_f32(int64_t N, const double* s, float4* s32, cudaStream_t st,
                         int64_t* launches) {
  k_to_f32<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, s, s32);
  ++*launches;
  return cudaGetLastError();
}

// Largest number of dipolar entries (exchange-only bonds excluded) in a row: Table 1's Delta.
__global__ void k_dip_degree(int64_t N, const uint32_t* __restrict__ row_ptr,
                             const uint32_t* __restrict__ col, DevCounters* __restrict__ cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  unsigned nd = 0;
  if (i < N)
    for (uint32_t e = row_ptr[i], e1 = row_ptr[i + 1]; e < e1; ++e)
      nd += (col[e] & kExchOnly) ? 0u : 1u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nd = max(nd, __shfl_down_sync(0xffffffffu, nd, o));
  if ((threadIdx.x & 31) == 0 && nd) atomicMax(&cnt->max_degree_dip, nd);
}

cudaError_t dip_degree_run(const DevParams& P, const uint32_t* row_ptr, const uint32_t* col,
                           DevCounters* cnt, cudaStream_t st, int64_t* launches) {
  cudaError_t e = cudaMemsetAsync(&cnt->max_degree_dip, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  k_dip_degree<<<(unsigned)((P.N + 255) / 256), 256, 0, st>>>(P.N, row_ptr, col, cnt);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t observables_run(const DevParams& P, const double* s, const uint32_t* row_ptr,
                            const uint32_t* col, const double2* xy, bool have_graph,
                            bool want_full, DevCounters* cnt, cudaStream_t st,
                            int64_t* launches) {
  cudaError_t e = cudaMemsetAsync(cnt->acc, 0, sizeof(cnt->acc), st);
  if (e != cudaSuccess) return e;
  const int nb = 4 * num_sms();
  k_site_obs<<<nb, 256, 0, st>>>(P, s, cnt->acc);
  ++*launches;
  if (have_graph) {
    k_pair_obs<<<nb, 256, 0, st>>>(P, s, row_ptr, col, xy, cnt->acc);
    ++*launches;
  }
  if (want_full) {
    k_full_energy<<<(unsigned)((P.N + 255) / 256), 256, 0, st>>>(P, s, cnt->acc);
    ++*launches;
  }
  return cudaGetLastError();
}

}  // namespace sco
