// stats.cu -- diagnostics of the switched graph and its colouring: the survival probability of a
// pair against its distance (Sec. 3.2, Fig. 5), the fraction of surviving pairs that join two
// cells of a virtual cell split of the lattice (Sec. 3.2, Fig. 6), and the colour-count imbalance
// Delta R of Eq. (9) over those cells (Sec. 3.3).  Counts are integers gathered by atomics (exact,
// order-free); the ratios are formed once, on the device, by the last kernel.
#include <cmath>
#include <cstdint>

#include "sco.h"
#include "sco_internal.h"

namespace sco {
namespace {

constexpr int kMaxBins = 4096;

// floor(sqrt(r2)) exactly: the rounded root corrected by integer comparisons.
__device__ __forceinline__ int64_t floor_sqrt(int64_t r2) {
  int64_t s = (int64_t)sqrt((double)r2);
  while (s * s > r2) --s;
  while ((s + 1) * (s + 1) <= r2) ++s;
  return s;
}

// Distance shell of a pair: bin b holds b + 1 <= r < b + 2, the last bin everything beyond.
__device__ __forceinline__ int shell_bin(int64_t r2, int nb) {
  const int64_t b = floor_sqrt(r2) - 1;
  return (int)(b < nb - 1 ? b : nb - 1);
}

// Cell of site (x, y) in a cx x cy split of the lattice into rectangles.
__device__ __forceinline__ uint32_t cell_of(uint32_t x, uint32_t y, const DevParams& P, int cx,
                                            int cy) {
  return (uint32_t)(((uint64_t)x * cx) / P.Lx + (uint64_t)cx * (((uint64_t)y * cy) / P.Ly));
}

// All site pairs of the open lattice per shell: displacement d of the half plane stands for the
// (Lx - |dx|)(Ly - |dy|) pairs (i, i + d) inside the lattice.
__global__ void __launch_bounds__(256) k_pair_shells(const DevParams P, const uint32_t* __restrict__ disp,
                                                     int nb, unsigned long long* __restrict__ pairs) {
  __shared__ unsigned long long h[kMaxBins];
  for (int b = threadIdx.x; b < nb; b += blockDim.x) h[b] = 0;
  __syncthreads();
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < P.K;
       m += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t d = disp[m];
    const int64_t dx = (int16_t)(d & 0xFFFFu), dy = d >> 16;
    const int64_t ax = dx < 0 ? -dx : dx;
    atomicAdd(&h[shell_bin(dx * dx + dy * dy, nb)],
              (unsigned long long)((P.Lx - ax) * (P.Ly - dy)));
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    if (h[b]) atomicAdd(&pairs[b], h[b]);
}

// Surviving dipolar pairs per shell and those whose sites lie in different cells: each pair is
// taken from the row of its smaller site (j > i), exchange-only bonds skipped.
__global__ void __launch_bounds__(256) k_edge_stats(const DevParams P, const uint32_t* __restrict__ row_ptr,
                                                    const uint32_t* __restrict__ col, int nb, int cx,
                                                    int cy, unsigned long long* __restrict__ surv,
                                                    unsigned long long* __restrict__ cross) {
  __shared__ unsigned int h[kMaxBins];
  for (int b = threadIdx.x; b < nb; b += blockDim.x) h[b] = 0;
  __syncthreads();
  unsigned long long nc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t yi = site_row((uint32_t)i, P), xi = (uint32_t)i - yi * (uint32_t)P.Lx;
    const uint32_t ci = cell_of(xi, yi, P, cx, cy);
    for (uint32_t e = row_ptr[i], e1 = row_ptr[i + 1]; e < e1; ++e) {
      const uint32_t cj = col[e];
      if ((cj & kExchOnly) || (int64_t)cj <= i) continue;
      const uint32_t yj = site_row(cj, P), xj = cj - yj * (uint32_t)P.Lx;
      const int64_t dx = (int64_t)xj - xi, dy = (int64_t)yj - yi;
      atomicAdd(&h[shell_bin(dx * dx + dy * dy, nb)], 1u);
      nc += cell_of(xj, yj, P, cx, cy) != ci;
    }
  }
  nc = warp_sum_u64(nc);
  if ((threadIdx.x & 31) == 0 && nc) atomicAdd(cross, nc);
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    if (h[b]) atomicAdd(&surv[b], (unsigned long long)h[b]);
}

// Sites of every colour in every cell: counts[colour * ncell + cell].
__global__ void __launch_bounds__(256) k_colour_cells(const DevParams P, const uint32_t* __restrict__ colour,
                                                      uint32_t g, int cx, int cy,
                                                      unsigned int* __restrict__ counts) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= P.N) return;
  const uint32_t y = site_row((uint32_t)i, P), x = (uint32_t)i - y * (uint32_t)P.Lx;
  const uint32_t c = colour[i];
  if (c < g) atomicAdd(&counts[(uint64_t)c * cx * cy + cell_of(x, y, P, cx, cy)], 1u);
}

// One block: Eq. (9) per colour (thread per colour, loop over the cells), then the mean and
// maximum over the non-empty colours, the survival fractions and P_IPC.
__global__ void __launch_bounds__(256) k_stats_final(uint32_t g, int64_t ncell, int nb,
                                                     const unsigned int* __restrict__ counts,
                                                     const unsigned long long* __restrict__ surv,
                                                     const unsigned long long* __restrict__ pairs,
                                                     const unsigned long long* __restrict__ cross,
                                                     double* __restrict__ delta_r,
                                                     double* __restrict__ p_survive,
                                                     double* __restrict__ summary) {
  __shared__ double s_sum[256], s_max[256];
  __shared__ unsigned long long s_ne[256], s_np[256], s_km[256], s_nt[256];
  double sum = 0.0, mx = 0.0;
  unsigned long long ne = 0, np = 0, km = 0, nt = 0;
  for (uint32_t c = threadIdx.x; c < g; c += blockDim.x) {
    unsigned long long tot = 0, kmax = 0;
    for (int64_t q = 0; q < ncell; ++q) {
      const unsigned long long k = counts[(int64_t)c * ncell + q];
      tot += k;
      kmax = k > kmax ? k : kmax;
    }
    km += kmax;
    nt += tot;
    double dr = __longlong_as_double(0x7FF8000000000000ll);  // NaN: empty colour
    if (tot > 0) {
      const double kave = (double)tot / (double)ncell;
      dr = ((double)kmax - kave) / kave;
      sum += dr;
      mx = fmax(mx, dr);
      ++ne;
    }
    delta_r[c] = dr;
  }
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    p_survive[b] = pairs[b] > 0 ? (double)surv[b] / (double)pairs[b]
                                : __longlong_as_double(0x7FF8000000000000ll);
    np += surv[b];
  }
  s_sum[threadIdx.x] = sum;
  s_max[threadIdx.x] = mx;
  s_ne[threadIdx.x] = ne;
  s_np[threadIdx.x] = np;
  s_km[threadIdx.x] = km;
  s_nt[threadIdx.x] = nt;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, m = 0.0;
    unsigned long long n = 0, p = 0, kms = 0, nts = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      a += s_sum[t];
      m = fmax(m, s_max[t]);
      n += s_ne[t];
      p += s_np[t];
      kms += s_km[t];
      nts += s_nt[t];
    }
    summary[0] = (double)p;                                    // surviving dipolar pairs
    summary[1] = (double)*cross;                               // of which across cells
    summary[2] = p > 0 ? (double)*cross / (double)p : 0.0;     // P_IPC
    summary[3] = n > 0 ? a / (double)n : 0.0;                  // mean Delta R
    summary[4] = m;                                            // max Delta R
    summary[5] = (double)(kms * (unsigned long long)ncell) / (double)nts - 1.0;  // weighted
  }
}

}  // namespace

cudaError_t graph_stats_run(const DevParams& P, const uint32_t* disp, const uint32_t* row_ptr,
                            const uint32_t* col, const uint32_t* colour, uint32_t g, int cx,
                            int cy, int nb, cudaStream_t st, int64_t* launches,
                            unsigned long long* h_counts, double* h_out) {
  // device scratch: survived, pairs, cross (u64), summary, delta_r, p_survive (f64), counts
  const int64_t ncell = (int64_t)cx * cy;
  const size_t n64 = 2 * (size_t)nb + 1, nf = 6 + (size_t)g + nb;
  const size_t ncnt = (size_t)g * ncell;
  char* buf = nullptr;
  const size_t bytes = 8 * (n64 + nf) + 4 * ncnt;
  cudaError_t e = cudaMalloc(&buf, bytes);
  if (e != cudaSuccess) return e;
  unsigned long long* surv = reinterpret_cast<unsigned long long*>(buf);
  unsigned long long* pairs = surv + nb;
  unsigned long long* cross = pairs + nb;
  double* fout = reinterpret_cast<double*>(buf + 8 * n64);
  unsigned int* counts = reinterpret_cast<unsigned int*>(buf + 8 * (n64 + nf));
  e = cudaMemsetAsync(buf, 0, bytes, st);
  const unsigned grid = (unsigned)(4 * num_sms());
  if (e == cudaSuccess) {
    k_pair_shells<<<grid, 256, 0, st>>>(P, disp, nb, pairs);
    k_edge_stats<<<grid, 256, 0, st>>>(P, row_ptr, col, nb, cx, cy, surv, cross);
    k_colour_cells<<<(unsigned)((P.N + 255) / 256), 256, 0, st>>>(P, colour, g, cx, cy, counts);
    k_stats_final<<<1, 256, 0, st>>>(g, ncell, nb, counts, surv, pairs, cross, fout + 6,
                                     fout + 6 + g, fout);
    *launches += 4;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h_counts, surv, 8 * n64, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_out, fout, 8 * nf, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(buf);
  return e;
}

}  // namespace sco
