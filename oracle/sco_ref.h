/*
 * sco_ref.h -- the ORACLE for the parallelized stochastic cutoff (SCO) method.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, CPU-only C restatement of
 * the method of Endo, Toga and Sasaki, "Parallelized Stochastic Cutoff Method
 * for Long-Range Interacting Systems" (arXiv:1503.03295).  It exists to check
 * the CUDA library; nothing in the product links it.  Only tests, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant with the CUDA path.
 *
 * Parity status per function is stated beside each declaration ("pinned by"
 * names the independent check in tests/).
 *
 * Conventions (Sec. 3.1, Eq. (6)):
 *   open Lx x Ly square lattice, site i = x + Lx*y, r_i = (x, y);
 *   classical Heisenberg spins |S| = 1, stored as three FP64 arrays (SoA);
 *   H = -J sum_<ij> S_i.S_j + D sum_{i<j} [S_i.S_j/r^3 - 3 (S_i.r)(S_j.r)/r^5].
 * The SCO switching (Sec. 2.1, Eqs. (1)-(3)) acts on the dipolar term only.
 */
#ifndef SCO_REF_H
#define SCO_REF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define SCO_REF_OK 0
#define SCO_REF_EINVAL 1
#define SCO_REF_ENOMEM 2

/* Philox counter word 3 ("tag") per use of the random stream. */
#define SCO_REF_TAG_INIT 1u
#define SCO_REF_TAG_SWITCH 2u
#define SCO_REF_TAG_PROPOSE 3u
#define SCO_REF_TAG_DIRECT 4u
#define SCO_REF_TAG_PLAIN 5u

/* Bit 31 of a CSR column entry: the pair is a nearest-neighbour exchange bond
 * whose dipolar potential was switched to zero (colouring only). */
#define SCO_REF_EXCH_ONLY 0x80000000u

typedef struct {
  int32_t Lx, Ly;         /* lattice size, >= 1 each, N = Lx*Ly >= 1 */
  double J;               /* exchange constant (any sign) */
  double D;               /* dipolar constant, >= 0 */
  double T;               /* temperature, > 0; beta = fl(1/T) */
  uint64_t seed;          /* Philox key word 0 */
  int32_t n_sw;           /* switch + colour every n_sw MC steps (Sec. 2.1 step B) */
  int32_t colour_variant; /* 0: KW over modified BCR (2)'; 1: KW over plain BCR (2) */
  int32_t replica;        /* Philox key word 1 */
  int32_t pad;
} sco_ref_params;

typedef struct {
  double e_switched;  /* H' of Eq. (4): sum of pseudointeractions over surviving pairs (+ exchange) */
  double e_exchange;  /* -J sum_<ij> S_i.S_j */
  double e_full;      /* full H of Eq. (6), NaN when not requested */
  double mx, my, mz;  /* magnetisation per spin */
  double m_abs;       /* |m| */
  double m_phi;       /* signed circular magnetisation inside |.| of Eq. (7) */
  int64_t n_edges;    /* surviving dipolar pairs */
  int32_t max_degree; /* Delta of the colouring graph */
  int32_t n_colours;  /* non-empty colour classes */
  int32_t kw_rounds;  /* running time t_R of the colouring (Sec. 2.3.1) */
  int32_t max_degree_dipolar; /* Delta over dipolar surviving pairs only (Table 1) */
  int64_t sweeps_done;
  int64_t guard_hits; /* decisions re-evaluated in extended precision */
} sco_ref_obs;

typedef struct sco_ref_ctx sco_ref_ctx;

/* ---- random numbers (ref_rng.c) ------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Pinned by: numpy.random.Philox. */
void sco_ref_philox(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
/* Marsaglia (1972) point on the sphere from two words; returns 1 on success.
 * Pinned by: moments <S>=0, <S_a S_b> = delta_ab/3, |S| = 1. */
int sco_ref_marsaglia(uint64_t w0, uint64_t w1, double S[3]);

/* ---- coupling table (ref_model.c) ------------------------------------------------ */
int64_t sco_ref_table_size(int32_t Lx, int32_t Ly);
/* Half-plane displacements sorted by (r^2, dy, dx) with c_m, hazard A_m, prefix W_m.
 * Pinned by: c vs r^-5, A*2^-59 >= 2/r^3 (exact rationals), counting of pairs. */
int sco_ref_table(int32_t Lx, int32_t Ly, int32_t* dx, int32_t* dy, int64_t* r2,
                  double* c, uint64_t* A, uint64_t* W);
/* Dipolar pair potential V_ij (Eq. (6)) for displacement (dx, dy) from i to j. */
double sco_ref_pair_V(double D, const double Si[3], const double Sj[3], int32_t dx, int32_t dy);
/* V_max of the pair at squared distance r2: D * A(r2) * 2^-59 (>= 2D/r^3). */
double sco_ref_vmax(double D, int64_t r2);
/* Switching probability P_ij (Eq. (2)) and pseudointeraction Vbar_ij (Eq. (3)). */
double sco_ref_switch_prob(double beta, double V, double Vmax);
double sco_ref_pseudo(double beta, double V, double Vmax);

/* ---- the chain (ref_chain.c) ------------------------------------------------------ */
int sco_ref_init(const sco_ref_params* p, sco_ref_ctx** out);
void sco_ref_destroy(sco_ref_ctx* c);
int sco_ref_switch(sco_ref_ctx* c);                    /* step (A) + CSR */
/* Step (A) at an explicit epoch (statistical tests draw many graphs for one state). */
int sco_ref_switch_epoch(sco_ref_ctx* c, uint32_t epoch);
int sco_ref_colour(sco_ref_ctx* c, int32_t* n_colours); /* KW colouring + classes */
int sco_ref_sweep(sco_ref_ctx* c, int32_t n_mcs);       /* step (B), re-switching every n_sw */
/* n MC steps recording full energy per spin (Eq. (6)) and |m| after each. */
int sco_ref_run_series(sco_ref_ctx* c, int64_t n_mcs, double* e_per_spin, double* m_abs);
int sco_ref_observables(sco_ref_ctx* c, sco_ref_obs* o, int32_t want_full);
int64_t sco_ref_n_sites(const sco_ref_ctx* c);
int64_t sco_ref_n_entries(const sco_ref_ctx* c); /* CSR entries = 2 * (undirected edges) */
int64_t sco_ref_n_half_edges(const sco_ref_ctx* c);
int sco_ref_get_spins(const sco_ref_ctx* c, double* xyz);       /* SoA 3*N */
int sco_ref_set_spins(sco_ref_ctx* c, const double* xyz);
/* CSR (row_ptr N+1, col entries) and colours (N); any pointer may be NULL. */
int sco_ref_get_graph(const sco_ref_ctx* c, int64_t* row_ptr, uint32_t* col, int32_t* colour);
/* Surviving half-plane edges in generation order: i, j, table index m, flags
 * (bit0 dipolar survivor, bit1 exchange bond). */
int sco_ref_get_edges(const sco_ref_ctx* c, int64_t* i, int64_t* j, int64_t* m, int32_t* flags);
/* Sites sorted by (colour, index) and class offsets (Delta+2 entries). */
int sco_ref_get_classes(const sco_ref_ctx* c, int64_t* perm, int64_t* off);
/* Accept bit per site for the last MC step run (1 accepted, 0 rejected). */
int sco_ref_get_accepts(const sco_ref_ctx* c, uint8_t* acc);
int64_t sco_ref_sweeps_done(const sco_ref_ctx* c);
void sco_ref_set_threads(int32_t n); /* OpenMP threads (<= 0: library default) */
/* Scale of every FP64 error bound (1 = normal; huge = always extended precision). */
void sco_ref_set_guard_scale(double s);

/* Changes T (the cooling protocol of Sec. 3.1: the paper lowers T in steps, carrying the spins
 * over); the graph of the old T is dropped and the next MC step switches again at its epoch. */
int sco_ref_set_temperature(sco_ref_ctx* c, double T);

/* Graph diagnostics of the current switched graph and colouring.
 *  - P_survive(r) (Sec. 3.2, Fig. 5): per distance shell (bin b: b+1 <= r < b+2, the last bin
 *    open-ended), surviving dipolar pairs over all site pairs of the open lattice in it.
 *  - P_IPC (Sec. 3.2, Fig. 6): the fraction of surviving dipolar pairs whose two sites lie in
 *    different cells of a cells_x x cells_y split of the lattice (site (x, y) in cell
 *    (floor(x cells_x / Lx), floor(y cells_y / Ly))).
 *  - Delta R (Sec. 3.3, Eq. (9)) per colour: (K_max - K_ave) / K_ave over the cells, K the
 *    number of sites of that colour in a cell (NaN for an empty colour); mean and max over the
 *    non-empty colours.
 * Any of survived, pairs, p_survive (n_rbins each) and delta_r (palette) may be NULL.
 * Pinned by: brute-force pair counts, the closed-form survival probability for uniform spins,
 * one-cell and one-site-per-cell limits, numpy recounts of the edge list and colours. */
typedef struct {
  int64_t n_pairs;     /* surviving dipolar pairs */
  int64_t n_cross;     /* of which the two sites lie in different cells */
  double p_ipc;        /* n_cross / n_pairs (0 without pairs) */
  double delta_r_mean; /* mean of Eq. (9) over the non-empty colours */
  double delta_r_max;
  double delta_r_weighted; /* class-size-weighted mean: cells * sum_c K_max,c / N - 1 */
  int32_t n_cells;
  int32_t palette;
} sco_ref_gstats;
int sco_ref_graph_stats(const sco_ref_ctx* c, int32_t cells_x, int32_t cells_y, int32_t n_rbins,
                        sco_ref_gstats* out, int64_t* survived, int64_t* pairs,
                        double* p_survive, double* delta_r);

/* KW colouring (Sec. 2.3.3) of an arbitrary symmetric CSR graph; bit 31 of col is ignored.
 * Pinned by: validity, palette [0, Delta], t_R <= (Delta+1)M (Eq. (5)), brute force. */
int sco_ref_kw_colour_graph(int64_t N, const int64_t* row_ptr, const uint32_t* col,
                            int32_t variant, int32_t* colour, int32_t* rounds,
                            int32_t* max_degree);

/* ---- definitional samplers (ref_defn.c) -------------------------------------------- */
/* O(N^2) switch: every pair independently survives with probability 1 - P_ij (Eq. (1)),
 * Philox tag DIRECT, epoch e.  Writes survive[i*N + j] for i < j (N*N bytes). */
int sco_ref_direct_switch(const sco_ref_ctx* c, uint32_t epoch, uint8_t* survive);
/* Plain full-interaction single-spin Metropolis on H of Eq. (6), sequential site order,
 * uniform new-direction proposals (tag PLAIN).  Per MC step writes E/N and |m|. */
int sco_ref_plain_metropolis(const sco_ref_params* p, const double* xyz0, int64_t n_mcs,
                             double* e_per_spin, double* m_abs, double* xyz_out);
/* Full H of Eq. (6) by direct summation over all pairs. */
double sco_ref_full_energy(const sco_ref_params* p, const double* xyz);

#ifdef __cplusplus
}
#endif
#endif
