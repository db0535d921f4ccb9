/*
 * sco.h -- C ABI of the GB300 library for the per-sweep hot path of the parallelized
 * stochastic cutoff (SCO) method of Endo, Toga and Sasaki (arXiv:1503.03295).
 *
 * One lattice (or a batch of replicas) lives in an opaque context that owns every device
 * buffer.  All work is enqueued on the CUDA stream given at creation; calls return a
 * status and never abort.  Every step of the path runs in the library's own CUDA kernels
 * (compute capability 10.3, sm_103a); there is no CPU fallback: without a usable device
 * sco_init returns SCO_ECUDA.
 *
 * Model (Sec. 3.1, Eq. (6)): open Lx x Ly square lattice, site i = x + Lx*y at r_i = (x, y),
 * classical Heisenberg spins |S| = 1,
 *     H = -J sum_<ij> S_i.S_j + D sum_{i<j} [S_i.S_j / r^3 - 3 (S_i.r)(S_j.r) / r^5].
 * The SCO switching (Sec. 2.1, Eqs. (1)-(3)) acts on the dipolar term; nearest-neighbour
 * exchange bonds are always present and join the colouring graph when J != 0.
 *
 * Per MC step (Fig. 1): (1) switch every dipolar pair to 0 or to its pseudointeraction,
 * (2) colour the graph of surviving pairs (Kuhn-Wattenhofer, Sec. 2.3), (3) update all
 * sites of each colour at once (Metropolis, uniform new direction).  Random numbers come
 * from Philox4x64-10 keyed by (seed, replica) with counter (site, step or epoch, draw,
 * tag), so a trajectory is a pure function of the parameters.
 *
 * Layouts: spins are SoA, three arrays of N doubles (x then y then z).  Graph: CSR with
 * row_ptr (N + 1 uint32) and col (uint32); rows sorted by neighbour index; bit 31 of a col
 * entry marks an exchange bond whose dipolar pair was switched to zero.
 *
 * Errors: SCO_EINVAL for bad arguments (nothing changed); SCO_ECUDA when a CUDA call fails
 * (the context should be destroyed); SCO_ETIMEOUT / SCO_ECAPACITY are raised on the device
 * (bounded waits, fixed-size buffers), become sticky, and are returned by the next call
 * that synchronises (sco_sync, sco_colour with a non-NULL count, getters, observables).
 */
#ifndef SCO_H
#define SCO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SCO_OK = 0,
  SCO_EINVAL = 1,     /* invalid argument or size */
  SCO_ENOMEM = 2,     /* device allocation failed */
  SCO_ECUDA = 3,      /* a CUDA runtime call failed (or no device) */
  SCO_ETIMEOUT = 4,   /* a bounded device-side wait gave up */
  SCO_ESTATE = 5,     /* call not valid in the current state (e.g. bad checkpoint) */
  SCO_EGUARD = 6,     /* reserved */
  SCO_ECAPACITY = 7   /* a fixed-size device buffer overflowed */
} sco_status;

typedef enum { SCO_FP64 = 0, SCO_FP32_GUARDED = 1 } sco_precision;

typedef struct {
  int32_t Lx, Ly;         /* lattice, 1 <= Lx, Ly <= 32767, Lx*Ly < 2^30 */
  double J;               /* exchange constant */
  double D;               /* dipolar constant, >= 0 */
  double T;               /* temperature > 0; beta = fl(1/T) */
  uint64_t seed;          /* Philox key word 0 */
  int32_t n_sw;           /* switch + colour every n_sw MC steps (Sec. 2.1 step (B)), >= 1 */
  int32_t precision;      /* sco_precision */
  int32_t colour_variant; /* 0: KW over modified BCR (2)'; 1: KW over plain BCR (2) */
  int32_t replica;        /* Philox key word 1 */
} sco_params;

typedef struct {
  double e_switched; /* H' of Eq. (4) (pseudointeractions of surviving pairs) + exchange */
  double e_exchange; /* -J sum_<ij> S_i.S_j */
  double e_full;     /* full H of Eq. (6) by direct summation; NaN unless requested */
  double mx, my, mz; /* magnetisation per spin */
  double m_abs;      /* |m| */
  double m_phi;      /* signed [(1/N) sum S_i x (r_i - r_c)/|r_i - r_c|]_z of Eq. (7) */
  int64_t n_edges;   /* surviving dipolar pairs */
  int32_t max_degree;         /* Delta of the colouring graph */
  int32_t n_colours;          /* non-empty colour classes */
  int32_t kw_rounds;          /* running time t_R of the colouring (Sec. 2.3.1, Eq. (5)) */
  int32_t max_degree_dipolar; /* Delta over dipolar pairs only (as in Table 1) */
  int64_t sweeps_done;        /* MC steps done */
  int64_t guard_hits_fp64;    /* decisions re-evaluated in double-double */
  int64_t guard_hits_fp32;    /* FP32 decisions re-evaluated in FP64 */
  int64_t kernel_launches;    /* kernels launched by this context so far */
} sco_obs;

typedef struct sco_ctx sco_ctx;

/* Creates a lattice: builds the coupling table, allocates every buffer and draws the
 * initial spins (uniform on the sphere, Philox tag INIT).  stream: a cudaStream_t (NULL =
 * legacy default stream); the caller keeps it alive until sco_destroy.  On success *out
 * owns all device memory.  Synchronises once. */
sco_status sco_init(const sco_params* p, void* stream, sco_ctx** out);
void sco_destroy(sco_ctx* c);

/* Step (A), Sec. 2.1: switches every dipolar pair at epoch t / n_sw from the current spins
 * (Eqs. (1)-(2)) and compacts the survivors into the CSR graph.  Synchronises once (to
 * size the graph). */
sco_status sco_switch(sco_ctx* c);

/* Step (2) of Fig. 1, Sec. 2.3.3: Kuhn-Wattenhofer (Delta+1)-colouring of the current graph
 * and the colour classes.  Switches first if no graph exists.  n_colours may be NULL. */
sco_status sco_colour(sco_ctx* c, int32_t* n_colours);

/* Steps (B)-(C), Sec. 2.1: n_mcs MC steps; before step t, if the graph is not the one of
 * epoch t / n_sw, switch and colour again.  One MC step updates every site once. */
sco_status sco_sweep(sco_ctx* c, int32_t n_mcs);

/* Observables of the current state (Eqs. (4), (6), (7), Table 1).  want_full computes the
 * full H by O(N^2) direct summation (N <= 65536, else e_full = NaN).  Synchronises. */
sco_status sco_observables(sco_ctx* c, sco_obs* out, int32_t want_full);

/* Spin copies (SoA, 3*N doubles).  on_device != 0: xyz is a device pointer.  Synchronous. */
sco_status sco_get_spins(sco_ctx* c, double* xyz, int32_t on_device);
sco_status sco_set_spins(sco_ctx* c, const double* xyz, int32_t on_device);

/* Sizes: sites, CSR entries of the current graph (0 if none), max degree, colour count
 * (Delta + 1 palette size).  Any pointer may be NULL. */
sco_status sco_get_sizes(sco_ctx* c, int64_t* n_sites, int64_t* n_entries, int32_t* max_degree,
                         int32_t* palette);

/* Host copies of the graph: row_ptr (N + 1), col (n_entries), colour (N); NULL skips.  col
 * comes with every row sorted by neighbour index (the library keeps its own rows in an internal
 * order, which changes no result; the copy is sorted on the device first). */
sco_status sco_get_graph(sco_ctx* c, uint32_t* row_ptr, uint32_t* col, uint32_t* colour);

/* Host copies of the colour classes: perm (N sites grouped by colour: off[c] .. off[c+1] - 1
 * hold class c; inside a class, for palettes up to 12288 colours, sites come by tiles of 2048
 * consecutive sites and inside a tile by degree then index; above that the order inside a class
 * is unspecified) and off (palette + 1 offsets). */
sco_status sco_get_classes(sco_ctx* c, uint32_t* perm, uint32_t* off);

/* Accept bit per site of the last MC step (N bytes, host). */
sco_status sco_get_accepts(sco_ctx* c, uint8_t* acc);

/* Host copy of the sorted half-plane coupling table: dx, dy (K int32 each), hazard prefix
 * W (K uint64) and c(r^2) ~ r^-5 (K doubles); K = (Lx-1) + (Ly-1)(2Lx-1). */
sco_status sco_get_table(sco_ctx* c, int64_t* K, int32_t* dx, int32_t* dy, uint64_t* W,
                         double* cc);

/* Changes the temperature (the cooling protocol of Sec. 3.1 lowers T step by step and carries
 * the spins over): rebuilds the temperature-dependent tables and drops the switched graph,
 * which belonged to the old T; the next MC step switches and colours again (same epoch
 * number, so the random streams stay those of a lattice started at the new T from the same
 * spins and step).  T > 0 and finite, else SCO_EINVAL.  Synchronises. */
sco_status sco_set_temperature(sco_ctx* c, double T);

/* Graph diagnostics of the current switched graph and its colouring, computed on the device:
 *  - P_survive(r) (Sec. 3.2, Fig. 5): per distance shell, surviving dipolar pairs over all
 *    site pairs of the open lattice in it; bin b holds b + 1 <= r < b + 2, the last of the
 *    n_rbins bins (1 <= n_rbins <= 4096) everything beyond;
 *  - P_IPC (Sec. 3.2, Fig. 6): the fraction of surviving dipolar pairs whose two sites lie in
 *    different cells of a virtual cells_x x cells_y split of the lattice into rectangles, site
 *    (x, y) in cell (floor(x cells_x / Lx), floor(y cells_y / Ly)) (1 <= cells_x <= Lx,
 *    1 <= cells_y <= Ly, palette x cells <= 2^28);
 *  - Delta R (Sec. 3.3, Eq. (9)) per colour: (K_max - K_ave) / K_ave, K the number of sites of
 *    that colour in a cell and K_ave the class size over the number of cells (NaN for an empty
 *    colour), with its mean and maximum over the non-empty colours.
 * survived and pairs (int64, n_rbins), p_survive (n_rbins) and delta_r (palette = Delta + 1
 * entries) are host buffers; any may be NULL.  SCO_ESTATE before the first colouring.
 * Synchronises; allocates its device scratch for the call. */
typedef struct {
  int64_t n_pairs;     /* surviving dipolar pairs */
  int64_t n_cross;     /* of which the two sites lie in different cells */
  double p_ipc;        /* n_cross / n_pairs (0 without pairs) */
  double delta_r_mean; /* mean of Eq. (9) over the non-empty colours */
  double delta_r_max;  /* its maximum */
  double delta_r_weighted; /* Eq. (9) weighted by class size: cells * sum_c K_max,c / N - 1
                              (the sweep's time over cells against a balanced split, minus 1) */
  int32_t n_cells;     /* cells_x * cells_y */
  int32_t palette;     /* Delta + 1 */
} sco_graph_stats;
sco_status sco_get_graph_stats(sco_ctx* c, int32_t cells_x, int32_t cells_y, int32_t n_rbins,
                               sco_graph_stats* out, int64_t* survived, int64_t* pairs,
                               double* p_survive, double* delta_r);

/* Checkpoint: a byte blob holding the parameters, the step counter, the spins and (when the
 * current epoch started before the current step) the spins at the epoch start, from which
 * the epoch's graph is rebuilt.  sco_get_state with buf == NULL returns the size in *len.
 * Restoring then continuing is bit-identical to an uninterrupted run. */
sco_status sco_get_state(sco_ctx* c, void* buf, size_t* len);
sco_status sco_set_state(sco_ctx* c, const void* buf, size_t len);

/* Device time (ms) spent in each phase since the last reset, measured with CUDA events on
 * the context's stream when enabled: [0] switch + CSR, [1] colouring + classes,
 * [2] colour-class sweeps.  enable = 0 stops recording. */
sco_status sco_set_timing(sco_ctx* c, int32_t enable);
sco_status sco_get_timing(sco_ctx* c, double ms[3], int64_t calls[3]);

/* Allocation-free colouring.  The paper has no counterpart: this entry point exists for
 * callers that cannot let a library allocate device memory while they run, for example an
 * application whose device memory is entirely carved up by its own pool allocator, or a
 * time-critical loop that must not pay for cudaMalloc/cudaFree (cudaFree synchronises the
 * whole device) or risk an allocation failure half-way through.
 *
 * Colours the caller's symmetric CSR graph exactly as sco_colour does (same colours, same
 * t_R; bit 31 of col entries is ignored).  row_ptr (n + 1), col and colour (n) are device
 * pointers owned by the caller (col non-NULL even for a graph without edges); max_degree
 * and rounds are optional host pointers.  The
 * working memory is one fixed device array inside the library, sized for
 * n <= SCO_KW_STATIC_MAX_VERTICES (8 MiB + 512 B, held on every device that loads the
 * library until the process exits); larger n returns SCO_EINVAL before any device work.
 * The first call on a device also does a one-time set-up with that device current: it
 * looks up that array's device address (cudaGetSymbolAddress) and the launch occupancy.
 * Every call reuses the same array
 * (the control block is cleared on each call), so calls that overlap on the GPU, from any
 * stream or thread, race: serialise them.  Every call copies max_degree and t_R back to the
 * host and synchronises `stream` before it returns; it returns SCO_ETIMEOUT if a bounded
 * device-side wait gave up.  No allocation of any kind. */
#define SCO_KW_STATIC_MAX_VERTICES (1 << 20)
sco_status sco_kw_colour_static(const uint32_t* row_ptr, const uint32_t* col, int64_t n,
                                int32_t variant, uint32_t* colour, int32_t* max_degree,
                                int32_t* rounds, void* stream);

/* ---- Batched replicas ------------------------------------------------------------------
 * A batch holds n_replicas independent lattices (any sizes, temperatures, seeds, J, D; one
 * precision and one n_sw for all) that advance together: each phase of Fig. 1 (switch +
 * CSR, KW colouring, colour-class sweep) is one launch over every replica, the sweep is one
 * persistent cooperative kernel per MC step that walks the colours with grid barriers, and
 * no step needs the host, so runs of steps are replayed as CUDA graphs.  Replica r follows
 * exactly the trajectory of a single lattice created with p[r] (same decisions, bit-identical
 * spins), whatever the tuning.
 *
 * Sizes that depend on the switched graph (CSR entries, overflow half-edges, palette) are
 * checked on the device; a step that would overflow is abandoned before any spin changes
 * and repeated after the host has grown the buffers ("replan"), so results do not depend on
 * the initial sizes either. */
typedef struct sco_batch sco_batch;

/* Result-invariant launch choices (autotuned or set by hand). */
typedef struct {
  int32_t steps_per_graph;     /* MC steps per replayed CUDA graph, >= 1 */
  int32_t sweep_blocks_per_sm; /* resident blocks per SM of the persistent sweep, >= 1 */
  int32_t kw_blocks_per_sm;    /* resident blocks per SM of the KW level kernel, >= 1 */
  int32_t use_graph;           /* 1: capture and replay graphs; 0: launch directly */
  int32_t kw_schedule;         /* 0: all KW levels in one kernel, vertices bucketed by colour
                                  and reduced largest colour first (order of Sec. 2.3.2 (2));
                                  1: one kernel per level, each vertex recolours as soon as
                                  its larger neighbours are done (2)'.  Same colours. */
  int32_t kw_low;              /* first KW levels, while a group has at most kw_low_group vertices
                                  and g <= 64: 1: one block per group, internal edges staged
                                  in shared memory (rows when they do not fit); 2: one block
                                  per group, rows read at every level; 0: by the level
                                  kernels above.  Same colours and rounds. */
  int32_t kw_low_group;        /* group-size cap of those levels: 1024, 2048 or 4096 vertices
                                  (smaller: one level fewer, more blocks per SM) */
} sco_batch_tuning;

/* Creates a batch of n_replicas lattices from p[0 .. n_replicas-1] (1 <= n_replicas <= 1024,
 * total sites < 2^31; every p[r] valid for sco_init; precision and n_sw equal for all).
 * stream: a cudaStream_t, or NULL for a stream the batch creates and owns (the legacy
 * default stream cannot be captured into graphs).  Draws every replica's initial spins.
 * Synchronises. */
sco_status sco_batch_init(const sco_params* p, int32_t n_replicas, void* stream,
                          sco_batch** out);
void sco_batch_destroy(sco_batch* b);

/* n_mcs MC steps of every replica (switch + colour every n_sw steps, then the sweep).
 * Synchronises once at the end (and once per replan). */
sco_status sco_batch_run(sco_batch* b, int32_t n_mcs);

/* Times the candidate tunings on real MC steps (trial_steps per candidate and one warm-up;
 * the steps count as MC steps done, and results do not depend on the tuning), keeps the
 * fastest and returns it in *chosen (may be NULL). */
sco_status sco_batch_autotune(sco_batch* b, int32_t trial_steps, sco_batch_tuning* chosen);
sco_status sco_batch_set_tuning(sco_batch* b, const sco_batch_tuning* t);
sco_status sco_batch_get_tuning(sco_batch* b, sco_batch_tuning* t);

/* Per-replica access, 0 <= r < n_replicas; same meaning and layouts as the single-lattice
 * calls (spins SoA 3*N_r doubles, graph with replica-local indices). */
sco_status sco_batch_observables(sco_batch* b, int32_t r, sco_obs* out, int32_t want_full);
sco_status sco_batch_get_spins(sco_batch* b, int32_t r, double* xyz, int32_t on_device);
sco_status sco_batch_set_spins(sco_batch* b, int32_t r, const double* xyz, int32_t on_device);
sco_status sco_batch_get_sizes(sco_batch* b, int32_t r, int64_t* n_sites, int64_t* n_entries,
                               int32_t* max_degree, int32_t* palette);
sco_status sco_batch_get_graph(sco_batch* b, int32_t r, uint32_t* row_ptr, uint32_t* col,
                               uint32_t* colour);
sco_status sco_batch_get_accepts(sco_batch* b, int32_t r, uint8_t* acc);

/* Totals: sites, MC steps done, kernel launches enqueued, graph replays, replans.  Any
 * pointer may be NULL. */
sco_status sco_batch_info(sco_batch* b, int64_t* total_sites, int64_t* steps_done,
                          int64_t* launches, int64_t* graph_launches, int32_t* replans);

/* Waits for the batch's stream; returns the sticky device status. */
sco_status sco_batch_sync(sco_batch* b);

/* Changes replica r's temperature (the cooling protocol of Sec. 3.1, run for many replicas at
 * once).  Allowed only between MC steps t with t mod n_sw = 0 (else SCO_ESTATE), where every
 * replica switches again anyway, so the change takes effect with the next step's switch; the
 * replica then follows the trajectory of a single lattice given the same sco_set_temperature
 * calls at the same steps.  Drops the captured graphs.  Synchronises. */
sco_status sco_batch_set_temperature(sco_batch* b, int32_t r, double T);

/* The same bound for the batch's kernels (grid barriers of the persistent sweep and of the
 * colouring, neighbour waits); drops the captured graphs.  Synchronises. */
sco_status sco_batch_set_wait_limit(sco_batch* b, uint64_t ns);

/* Self-test of the library's own elementary function: the branch-free expm1 for x <= 0.35 used
 * by the FP64 decisions of the switch (argument reduction by ln 2, a degree-8
 * polynomial on |r| <= 0.35, -1 below x = -40), stated relative error bound 2^-42, which those
 * decisions carry in their error bounds.  Evaluates it at n >= 17 points of [-50, 0.35] (16
 * fixed points, then Philox-jittered evenly spaced ones from `seed`) and returns the largest
 * relative error against the library's double-double expm1 (max_rel_err) and against CUDA's
 * expm1 (max_rel_diff_cuda, may be NULL).  Synchronous; uses the current device.  There is no
 * counterpart in the paper. */
sco_status sco_selftest_expm1(int64_t n, uint64_t seed, double* max_rel_err,
                              double* max_rel_diff_cuda);

/* The same for either degree of the polynomial: degree 8 (the one above, used by the switch)
 * or degree 6 (used by the sweep decisions, stated relative error bound 2^-31).  Any other
 * degree: SCO_EINVAL. */
sco_status sco_selftest_expm1_deg(int64_t n, uint64_t seed, int32_t degree, double* max_rel_err,
                                  double* max_rel_diff_cuda);

/* Device self-test of the library's own natural logarithm for 0 < x <= 1, used by the FP64
 * candidate search of the switch (table-driven reduction, degree-4 polynomial; stated relative
 * error bound 2^-49, carried in that search's margin).  Evaluates it at n >= 17 points (16 fixed
 * ones, then Philox-drawn values over all octaves of (2^-53, 1) and just below 1, from `seed`)
 * and returns the largest relative error against the library's double-double log
 * (max_rel_err; at x = 1 the absolute value, 0 expected) and against CUDA's log
 * (max_rel_diff_cuda, may be NULL).  Synchronous; uses the current device. */
sco_status sco_selftest_log(int64_t n, uint64_t seed, double* max_rel_err,
                            double* max_rel_diff_cuda);

/* FP64 throughput probe of the current device (no counterpart in the paper; it measures the
 * peak that the FP64 forms of the switch and sweep are held against).  Three timed launches,
 * each filling every SM with resident 256-thread blocks whose threads advance 8 independent
 * chains: out[0] = FP64 FMA lane-operations per second (FLOP/s = 2 out[0]) over `iters` FMA
 * steps per chain; out[1] = evaluations per second of the library's expm1 (degree 6, the
 * sweep decisions' one) and out[2] of its log, each chain step being one evaluation plus one
 * FMA, over iters / 12 steps.  iters in [1, 2^30].  Synchronous, on the legacy default
 * stream of the current device; allocates 8 bytes. */
sco_status sco_probe_fp64(int64_t iters, double out[3]);

/* Waits for the context's stream; returns the sticky device status. */
sco_status sco_sync(sco_ctx* c);

/* Bound (ns) of every device-side wait of this context's kernels (the grid barriers and
 * neighbour waits of the colouring, Sec. 2.3.3); default 2 s, at most 1 h.  A wait that runs
 * past it gives up, the kernel returns, and SCO_ETIMEOUT becomes the context's sticky
 * status: sco_sync and every later call return it, and the context does no further work (it
 * must be destroyed).  Limits below 1 ms are checked on every spin of a wait.  Used by tests
 * of the failure path; there is no counterpart in the paper.  Synchronises. */
sco_status sco_set_wait_limit(sco_ctx* c, uint64_t ns);

const char* sco_strerror(sco_status s);

#ifdef __cplusplus
}
#endif
#endif
