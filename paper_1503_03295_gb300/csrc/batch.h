// batch.h -- device-side layout of a batch of independent replicas (lattices of any size,
// temperature, seed) that run the per-step path of Fig. 1 together: one launch per phase
// covers every replica, and no step needs the host (sizes that depend on the graph are read
// on the device), so a whole run of steps can be captured in one CUDA graph.
//
// Sites of all replicas are numbered globally: replica r owns sites [base_r, base_r + N_r).
// Spins of replica r are the SoA block s + 3 base_r (x, y, z arrays of N_r each).  CSR
// row_ptr holds global entry offsets; col entries are replica-local site indices (bit 31:
// exchange-only bond), so row_ptr + base_r with col is replica r's own CSR graph.
#pragma once

#include <cstdint>

#include "sco.h"
#include "sco_internal.h"

namespace sco {

constexpr int kMaxReplicas = 1024;
constexpr int kBatchBlock = 256;  // sites per block of the per-site batch kernels

// Constant description of replica r.
struct RepDesc {
  DevParams P;
  const uint64_t* W;  // hazard prefix of the lattice shape (shared between replicas)
  const uint32_t* disp;
  const double2* xy;
  const double* xyq;
  const float4* xy32;
  const Sw64* sw64;
  const float4* sw32;
  int32_t mnn0, mnn1;  // list index of the displacements (1, 0) and (0, 1)
  uint32_t base;       // first global site
  int32_t variant;     // colouring variant (reported t_R only)
};

// Larger right-half neighbours listed per bucketed vertex of the KW colouring (records).
constexpr int kKwItemList = 32;

// Per-step plan of replica r, written on the device once the graph is known.
struct RepPlan {
  uint32_t g;       // Delta + 1
  uint32_t levels;  // KW levels M
  unsigned long long magic;  // div_magic(g)
};

// Batch control word block (device).
struct BatchCtl {
  unsigned long long step;      // MC steps done by every replica
  unsigned long long nnz;       // CSR entries of all replicas (scan total)
  unsigned long long ovf_n;     // overflow half-edges of this switch
  unsigned long long need_col;  // CSR entries seen when col was too small
  int flag;                     // replan request (kReplan* bits): every kernel returns
  int ovf_full;                 // overflow list too small (set by the switch)
  int status;                   // sticky device error (sco_status), e.g. a wait gave up
  unsigned gmax;                // max palette over replicas this epoch
  unsigned lmax;                // max KW levels over replicas this epoch
  unsigned bar[2];              // grid barrier of the persistent kernels (count, generation)
  unsigned pad;
};
constexpr int kReplanCol = 1, kReplanOvf = 2, kReplanPal = 4;

// Device pointers and sizes of a batch (passed by value to every batch kernel).
struct BatchDev {
  const RepDesc* desc;
  RepPlan* plan;
  DevCounters* cnt;  // R per-replica counters
  BatchCtl* ctl;
  const uint32_t* blk_start;   // R + 1: first block of each replica in per-site launches
  const uint32_t* site_start;  // R + 1: global site bases (site_start[R] = Ntot)
  int R;
  uint32_t Ntot;
  uint32_t nblocks;  // blk_start[R]
  int precision;
  int n_sw;
  double* s;
  float4* s32;  // FP32 copy of the spins, one (x, y, z, 0) per site
  uint8_t* acc;
  uint32_t* hslot;
  uint32_t* hcnt;
  uint32_t* indeg;
  uint32_t* deg;  // Ntot + 1 (deg[Ntot] stays 0)
  uint32_t* lcur;
  uint32_t* ocur;
  uint32_t* ovf;
  uint32_t ovf_cap;
  uint32_t* row_ptr;  // Ntot + 1
  uint32_t* col;
  unsigned long long col_cap;
  unsigned long long* word;
  uint8_t* col8;  // colour (low byte) beside the words
  uint32_t* blk;
  uint32_t* colour;
  uint32_t* used;  // R * pal_cap / 32 colour-in-use bits
  uint32_t pal_cap;
  uint32_t ntiles;
  uint32_t* tile_cnt;  // pal_cap * ntiles + 1
  uint32_t* perm;      // Ntot, global sites sorted by (colour, global index)
  uint32_t* off;       // pal_cap + 1 class offsets
  uint32_t* defer;     // Ntot
  double4_32a* prop;   // Ntot proposals {S', u} of the current MC step
  uint32_t* dcnt;      // pal_cap
  uint32_t* bcnt;      // 32 x pal_cap KW bucket sizes per level
  unsigned long long* imask;  // Ntot per-level vertex records of the colouring kernel
  uint32_t* imeta;            // Ntot
  uint32_t* ilist;            // 8 Ntot (kItemList per record)
  unsigned long long ns_limit;  // bound of every device-side wait
};

// Parameter checks and the kernel parameter block of one lattice (api.cu).
bool params_ok(const sco_params* p);
DevParams make_dev_params(const sco_params& p);

// Launchers (batch.cu).  Each enqueues one phase for every replica on `st`.
struct BatchLaunch {
  int kw_schedule;  // 0: all levels in one kernel, buckets by colour; 1: one async kernel per level
  int kw_low;       // 0: no block-local levels; 1: staged edges; 2: rows at every level
  uint32_t low_gmax;  // group-size cap of the block-local levels
  int low_grid;     // blocks of the block-local level kernel
  uint32_t low_ecap;  // its staged-edge capacity per group
  int kw_grid;     // blocks of the persistent KW kernel(s)
  int sweep_grid;  // blocks of the persistent sweep kernel
  unsigned levels;  // KW level launches per colouring (>= every replica's M)
  uint64_t* scan_tmp;
  int64_t* launches;
};
cudaError_t batch_switch(const BatchDev& B, const BatchLaunch& L, cudaStream_t st);
cudaError_t batch_colour(const BatchDev& B, const BatchLaunch& L, cudaStream_t st);
cudaError_t batch_sweep(const BatchDev& B, const BatchLaunch& L, cudaStream_t st);
cudaError_t batch_step_end(const BatchDev& B, const BatchLaunch& L, cudaStream_t st);
// co-resident blocks per SM of the two persistent kernels (for the grid sizes)
int batch_kw_occupancy(int schedule, int R, unsigned pal);
// blocks per SM of the block-local level kernel and its staged-edge capacity (sets the
// kernel's shared-memory limit)
cudaError_t batch_low_setup(int R, uint32_t gcap, int* blocks_per_sm, uint32_t* ecap);
int batch_sweep_occupancy(int precision, int R);
size_t batch_sweep_smem(int R);

}  // namespace sco
