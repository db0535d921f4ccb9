// sco_internal.h -- host-side declarations shared by the CUDA translation units of the
// SCO library: the launchers each .cu file exports to the C-ABI layer (api.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "sco_device.cuh"

namespace sco {

// Device-resident counters of one lattice (one struct per replica).
struct DevCounters {
  unsigned long long n_half;        // surviving half-plane pairs incl. exchange-only bonds
  unsigned long long n_dip;         // surviving dipolar pairs
  unsigned long long ovf_n;         // half-edges beyond the per-site slots
  unsigned long long nnz;           // CSR entries
  unsigned long long guard_fp64;    // decisions re-evaluated in double-double
  unsigned long long guard_fp32;    // decisions re-evaluated in FP64 (FP32-guarded form)
  unsigned int max_degree;          // Delta of the colouring graph
  unsigned int max_degree_dip;      // Delta over dipolar pairs
  unsigned int g;                   // Delta + 1
  unsigned int levels;              // KW levels M
  unsigned int kw_rounds;           // t_R (sum over levels of the deepest dependency chain)
  unsigned int n_colours;           // non-empty classes
  int status;                       // sticky device error (sco_status value), 0 if none
  int ovf_full;                     // the switch wrote more half-edges than the overflow list holds
  double acc[8];                    // observable accumulators
  unsigned int lev_rounds[32];      // deepest dependency chain per KW level
  unsigned int bar[2];              // grid barrier of the persistent colouring kernel
  unsigned int sw_next;             // next unclaimed site of the persistent switch kernel
};

// ---- scan.cu ----
size_t scan_tmp_bytes(int64_t n);
cudaError_t scan_excl_u32(const uint32_t* in, uint32_t* out, int64_t n, uint64_t* tmp,
                          uint64_t* total_dev, cudaStream_t s, int64_t* launches);
cudaError_t scan_incl_u64(const uint64_t* in, uint64_t* out, int64_t n, uint64_t* tmp,
                          uint64_t* total_dev, cudaStream_t s, int64_t* launches);

// ---- table.cu ----
struct Table {
  int64_t K = 0;
  uint32_t* disp = nullptr;  // packed (dx & 0xFFFF) | (dy << 16), sorted by (r^2, dy, dx)
  uint64_t* W = nullptr;     // inclusive prefix of the integer hazards A_m
  // by list index m: the bits of fl(exp(-beta D 2^-58 W_m)), the probability that a walk from
  // the list's start passes m without a candidate (FP64 candidate search; temperature-dependent,
  // built with the tables by (|dx|, |dy|) once the list exists)
  uint64_t* Ebits = nullptr;
  double2* xy = nullptr;     // by (|dx|, |dy|): {fl(D c(r^2)), V_max = fl(fl(D A) 2^-59)}
  double* xyq = nullptr;     // by (|dx|, |dy|): q = -expm1(-2 beta V_max), candidate probability
  float4* xy32 = nullptr;    // by (|dx|, |dy|): FP32 copies {Dc, Vmax, 2 beta Vmax, q}
  Sw64* sw64 = nullptr;      // sweep, by (|dx|, |dy|): FP64 decision constants (see Sw64)
  float4* sw32 = nullptr;    // the same in FP32 (with its own c0)
  int32_t m_nn[2] = {-1, -1};
};
cudaError_t table_build(const DevParams& P, Table& t, cudaStream_t s, int64_t* launches);
// the two halves: the temperature-dependent tables by (|dx|, |dy|), and the sorted list
// with its hazard prefix (depends on Lx, Ly only; synchronises)
cudaError_t table_build_xy(const DevParams& P, Table& t, cudaStream_t s, int64_t* launches);
cudaError_t table_build_list(const DevParams& P, Table& t, cudaStream_t s, int64_t* launches);
void table_free(Table& t);
void table_free_xy(Table& t);

// ---- init / observables (spins.cu) ----
cudaError_t spins_init(const DevParams& P, double* s, float4* s32, cudaStream_t st,
                       int64_t* launches);
cudaError_t spins_to_f32(int64_t N, const double* s, float4* s32, cudaStream_t st,
                         int64_t* launches);
// largest dipolar degree of the current graph into cnt->max_degree_dip
cudaError_t dip_degree_run(const DevParams& P, const uint32_t* row_ptr, const uint32_t* col,
                           DevCounters* cnt, cudaStream_t st, int64_t* launches);
cudaError_t observables_run(const DevParams& P, const double* s, const uint32_t* row_ptr,
                            const uint32_t* col, const double2* xy, bool have_graph,
                            bool want_full, DevCounters* cnt, cudaStream_t st, int64_t* launches);

// ---- switch.cu ----
constexpr int kSlotCap = 32;
struct SwitchBufs {
  uint32_t* hslot;  // N * kSlotCap upper neighbours (j | flag) per site
  uint32_t* hcnt;   // N half-degree per site
  uint32_t* indeg;  // N lower-neighbour count per site (also the fill cursor base)
  uint32_t* deg;    // N + 1
  uint32_t* lcur;   // N lower fill cursor
  uint32_t* ocur;   // N overflow fill cursor
  uint32_t* ovf;    // 2 * ovf_cap (i, j | flag)
  uint32_t ovf_cap;
  uint64_t* scan_tmp;
  // FP64 form only (else null): the pair cache, one 32-byte record per half-edge id h (slot
  // i * kSlotCap + q of site i, then N * kSlotCap + overflow index), N * kSlotCap + ovf_cap of
  // them, two halves of {1 - P_ij, x = beta (V - Vmax)}: one holds the pair at the current
  // spins, the other the pair after the last proposed move of one endpoint (which half is which
  // follows the endpoints' acceptance parities, see PairCache), so that every access of a pair
  // touches one sector.  The switch writes the first half.
  double4_32a* keep;
};
cudaError_t switch_run(const DevParams& P, const Table& t, const double* s, const float4* s32,
                       int precision, uint32_t epoch, SwitchBufs& b, DevCounters* cnt,
                       cudaStream_t st, int64_t* launches);
cudaError_t csr_scan(const DevParams& P, SwitchBufs& b, uint32_t* row_ptr, DevCounters* cnt,
                     cudaStream_t st, int64_t* launches);
// hid (optional, parallel to col): the half-edge id of every CSR entry (both entries of a pair
// carry the id of its half-edge).  sort_rows (only without hid): sort every row by neighbour
// index and record the largest dipolar degree; else a row holds its lower neighbours in the
// order of their atomic slots, then its upper ones in switching order (no result depends on
// the order inside a row).
cudaError_t csr_fill(const DevParams& P, const SwitchBufs& b, const uint32_t* row_ptr,
                     uint32_t* col, uint32_t* hid, bool has_overflow, bool sort_rows,
                     DevCounters* cnt, cudaStream_t st, int64_t* launches);
// out = col with every row sorted by neighbour index (the documented layout of the getters);
// also records the largest dipolar degree in cnt.
cudaError_t csr_sorted_copy(const DevParams& P, const uint32_t* row_ptr, const uint32_t* col,
                            uint32_t* out, uint64_t nnz, DevCounters* cnt, cudaStream_t st,
                            int64_t* launches);

// ---- colour.cu ----
struct ColourBufs {
  unsigned long long* word;  // N packed (level tag, round, colour)
  uint8_t* col8;     // N colour (low byte), kept beside the words for the neighbour gathers
  uint32_t* blk;     // N neighbour each unfinished vertex waits for (0xFFFFFFFF: none)
  uint32_t* colour;  // N final colours
  uint32_t* hist;    // g + 1
  uint32_t* off;     // g + 1
  uint32_t* cursor;  // g
  uint32_t* dcnt;    // g deferred sweep decisions per colour
  uint32_t* perm;    // N
  uint32_t* tile_cnt;  // (colour, tile, degree bin) counts (+1), scanned in place
  uint64_t* scan_tmp;
  uint32_t* bcnt;    // 32 x palette KW bucket sizes per level
  uint32_t* meta;    // 6 words: one-lattice view of the persistent colouring kernel
  unsigned long long* imask;  // N per-level vertex records of the colouring kernel
  uint32_t* imeta;            // N
  uint32_t* ilist;            // 32 N (kItemList per record)
  uint32_t* boff;             // kKwSplitBlocks x 64: per (block, colour) bucket offsets of the
                              // split record build (null: records built inside k_kw_bcr)
};
constexpr int kKwSplitBlocks = 2048;
constexpr uint32_t kMaxStablePalette = 12288;  // palettes up to this size get stable classes
constexpr int64_t kClassTileSites = 2048;
// ns_limit: bound of every device-side wait of the colouring kernels (SCO_ETIMEOUT after it)
cudaError_t kw_run(const DevParams& P, const uint32_t* row_ptr, const uint32_t* col,
                   uint32_t g, int variant, ColourBufs& b, DevCounters* cnt,
                   unsigned long long ns_limit, cudaStream_t st, int64_t* launches);
cudaError_t bucket_run(const DevParams& P, uint32_t g, const uint32_t* row_ptr, ColourBufs& b,
                       DevCounters* cnt, cudaStream_t st, int64_t* launches);

// ---- sweep.cu ----
// The FP64 form's pair cache (see sweep_dev.cuh); hid null: no cache.
struct PairCache {
  const uint32_t* hid;  // per CSR entry: half-edge id of its pair
  double4_32a* keep;    // per half-edge: the two halves of SwitchBufs::keep
  // per site: bit 2 the parity p_i of its accepted moves since the halves were last written
  // from the spins (the switch, or cache_build_run), bits 0-1 its decision in this MC step
  // (0 not decided, 1 rejected, 2 accepted); an accepted move flips p_i as it is decided.  The
  // current terms of pair (i, j) are in half p_i ^ p_j (0 after a reset): a site reads that
  // half and writes its proposed-spin terms into the other, so an acceptance flips the half.
  uint8_t* upd;
  int carry;  // the next step uses this graph again: the endpoint decided last writes too
  int reset;  // the halves were written from the spins: every parity starts at 0
};
cudaError_t sweep_run(const DevParams& P, const Table& t, double* s, float4* s32,
                      const uint32_t* row_ptr, const uint32_t* col, const uint32_t* perm,
                      const uint32_t* off, uint32_t g, uint64_t step, int precision,
                      uint8_t* acc, uint32_t* defer, uint32_t* dcnt, double4_32a* prop,
                      DevCounters* cnt, const PairCache& pc, cudaStream_t st,
                      int64_t* launches);
// Between two MC steps on the same graph after the spins changed outside the sweep: the pair
// cache rebuilt from the spins (first halves; the next sweep resets the parities).
cudaError_t cache_build_run(const DevParams& P, const Table& t, const double* s,
                            const SwitchBufs& b, const DevCounters* cnt, cudaStream_t st,
                            int64_t* launches);

// ---- stats.cu ----
// Graph diagnostics (see sco_get_graph_stats); copies 2 nb + 1 counts (survived, pairs, cross)
// to h_counts and 6 + g + nb doubles (summary, Delta R per colour, P_survive) to h_out, then
// synchronises.
cudaError_t graph_stats_run(const DevParams& P, const uint32_t* disp, const uint32_t* row_ptr,
                            const uint32_t* col, const uint32_t* colour, uint32_t g, int cx,
                            int cy, int nb, cudaStream_t st, int64_t* launches,
                            unsigned long long* h_counts, double* h_out);

int num_sms();

}  // namespace sco
