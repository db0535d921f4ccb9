/*
 * ref_chain.c -- the oracle's SCO chain: initial spins, potential switching
 * (step (A)), the interaction graph, Kuhn-Wattenhofer colouring, colour-class
 * Metropolis steps (step (B)) and observables.  TEST INFRASTRUCTURE ONLY.
 *
 * Every random decision is defined as an exact comparison of real numbers
 * computed from FP64 inputs (spins, c(r^2), A(r^2), beta = fl(1/T), D, J and the
 * uniforms).  The oracle evaluates it in FP64 together with an upper bound of
 * the FP64 error; when the FP64 margin does not exceed the bound, the decision
 * is taken again in extended precision (long double) and counted as a guard hit.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "ref_internal.h"

struct sco_ref_ctx {
  sco_ref_params p;
  int64_t N;
  double beta; /* fl(1/T) */
  double bD;   /* fl(beta * D) */
  /* coupling table, sorted half-plane displacements */
  int64_t K;
  int32_t *tdx, *tdy;
  int64_t* tr2;
  double* tc;
  uint64_t *tA, *tW;
  int64_t m_nn[2]; /* table index of (1,0) and (0,1), -1 if absent */
  /* spins, SoA */
  double* s;
  /* surviving half-plane edges in generation order */
  int64_t ne;
  int32_t *ei, *ej, *em, *ef;
  /* graph */
  int64_t* row_ptr;
  uint32_t* col;
  int64_t nnz;
  int32_t max_degree, max_degree_dip;
  /* colouring */
  int32_t* colour;
  int32_t kw_rounds;
  int32_t g;
  int64_t *perm, *off;
  uint8_t* acc;
  /* chain state */
  int64_t t;
  int64_t graph_epoch;
  int colour_valid;
  int64_t guard_hits;
};

static inline void spin_get(const sco_ref_ctx* c, int64_t i, double S[3]) {
  S[0] = c->s[i];
  S[1] = c->s[c->N + i];
  S[2] = c->s[2 * c->N + i];
}

static inline void draw(const sco_ref_ctx* c, uint64_t site, uint64_t step, uint64_t a,
                        uint64_t tag, uint64_t w[4]) {
  uint64_t ctr[4] = {site, step, a, tag};
  uint64_t key[2] = {c->p.seed, (uint64_t)(uint32_t)c->p.replica};
  sco_ref_philox(ctr, key, w);
}

/* Multiplies every FP64 error bound; tests set it huge to send every decision through the
 * extended-precision path and check that the trajectory does not change. */
static double g_guard_scale = 1.0;
void sco_ref_set_guard_scale(double s) { g_guard_scale = s > 0 ? s : 1.0; }

static inline double unif(uint64_t w) { return (double)(w >> 11) * 0x1p-53; }
static inline double unif_pos(uint64_t w) { return ((double)(w >> 11) + 1.0) * 0x1p-53; }

void sco_ref_set_threads(int32_t n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ---- lifetime -------------------------------------------------------------------- */
static void free_graph(sco_ref_ctx* c) {
  free(c->ei); free(c->ej); free(c->em); free(c->ef);
  free(c->row_ptr); free(c->col);
  c->ei = c->ej = c->em = c->ef = NULL;
  c->row_ptr = NULL;
  c->col = NULL;
  c->ne = c->nnz = 0;
}

void sco_ref_destroy(sco_ref_ctx* c) {
  if (!c) return;
  free_graph(c);
  free(c->tdx); free(c->tdy); free(c->tr2); free(c->tc); free(c->tA); free(c->tW);
  free(c->s); free(c->colour); free(c->perm); free(c->off); free(c->acc);
  free(c);
}

int sco_ref_init(const sco_ref_params* p, sco_ref_ctx** out) {
  if (!p || !out) return SCO_REF_EINVAL;
  *out = NULL;
  if (p->Lx < 1 || p->Ly < 1 || !(p->T > 0) || !(p->D >= 0) || !isfinite(p->J) ||
      !isfinite(p->D) || p->n_sw < 1 || p->colour_variant < 0 || p->colour_variant > 1)
    return SCO_REF_EINVAL;
  if ((int64_t)p->Lx * p->Ly >= (1ll << 31)) return SCO_REF_EINVAL;
  sco_ref_ctx* c = (sco_ref_ctx*)calloc(1, sizeof(sco_ref_ctx));
  if (!c) return SCO_REF_ENOMEM;
  c->p = *p;
  c->N = (int64_t)p->Lx * p->Ly;
  c->beta = 1.0 / p->T;
  c->bD = c->beta * p->D;
  c->K = sco_ref_table_size(p->Lx, p->Ly);
  int64_t K = c->K > 0 ? c->K : 1;
  c->tdx = (int32_t*)malloc(K * sizeof(int32_t));
  c->tdy = (int32_t*)malloc(K * sizeof(int32_t));
  c->tr2 = (int64_t*)malloc(K * sizeof(int64_t));
  c->tc = (double*)malloc(K * sizeof(double));
  c->tA = (uint64_t*)malloc(K * sizeof(uint64_t));
  c->tW = (uint64_t*)malloc(K * sizeof(uint64_t));
  c->s = (double*)malloc(3 * c->N * sizeof(double));
  c->colour = (int32_t*)calloc(c->N, sizeof(int32_t));
  c->perm = (int64_t*)malloc(c->N * sizeof(int64_t));
  c->acc = (uint8_t*)calloc(c->N, 1);
  if (!c->tdx || !c->tdy || !c->tr2 || !c->tc || !c->tA || !c->tW || !c->s || !c->colour ||
      !c->perm || !c->acc) {
    sco_ref_destroy(c);
    return SCO_REF_ENOMEM;
  }
  sco_ref_table(p->Lx, p->Ly, c->tdx, c->tdy, c->tr2, c->tc, c->tA, c->tW);
  c->m_nn[0] = c->m_nn[1] = -1;
  for (int64_t m = 0; m < c->K && m < 2; ++m) {
    if (c->tdx[m] == 1 && c->tdy[m] == 0) c->m_nn[0] = m;
    if (c->tdx[m] == 0 && c->tdy[m] == 1) c->m_nn[1] = m;
  }
  /* initial spins: uniform on the sphere, Philox tag INIT, attempt a = 0..63 */
  const int64_t N = c->N;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; ++i) {
    double S[3] = {0.0, 0.0, 1.0};
    for (uint64_t a = 0; a < 64; ++a) {
      uint64_t w[4];
      draw(c, (uint64_t)i, 0, a, SCO_REF_TAG_INIT, w);
      if (sco_ref_marsaglia(w[0], w[1], S)) break;
      S[0] = 0.0; S[1] = 0.0; S[2] = 1.0;
    }
    c->s[i] = S[0];
    c->s[N + i] = S[1];
    c->s[2 * N + i] = S[2];
  }
  c->graph_epoch = -1;
  c->colour_valid = 0;
  *out = c;
  return SCO_REF_OK;
}

/* ---- step (A): switching ----------------------------------------------------------- */
/* Sec. 2.1 (A) switches every pair independently: it survives (V -> Vbar) with
 * probability 1 - P_ij.  Testing every pair costs O(N^2); the method relies on an
 * O(N) technique whose details are in a reference that is not reproduced here.
 * The oracle uses bound thinning: element m of the half-plane list is made a
 * candidate with probability q_m = 1 - exp(-2 beta V_max,m) >= 1 - P_ij, by a
 * Poisson process of rate 2 beta V_max,m = beta D A_m 2^-58 per element run over
 * the prefix sums W_m, and a candidate survives with probability (1 - P_ij) / q_m.
 * The product is exactly 1 - P_ij per pair, independently across pairs. */

/* Next candidate after s: min { k > s : beta D 2^-58 (W_k - W_s) >= -ln u+ }, K if none. */
static int64_t next_candidate(const sco_ref_ctx* c, int64_t s, uint64_t wE, int64_t* guard) {
  const uint64_t* W = c->tW;
  const int64_t K = c->K;
  if (K == 0 || s >= K - 1) return K;
  if (!(c->bD > 0.0)) return K;
  const uint64_t Ws = s >= 0 ? W[s] : 0;
  const double up = unif_pos(wE);
  const double tau = (-log(up) / c->bD) * 0x1p58;
  int64_t lo = s + 1, hi = K;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if ((double)(W[mid] - Ws) >= tau) hi = mid; else lo = mid + 1;
  }
  const int64_t k = lo;
  /* tau carries < 2^-49 relative error (log, one division, fl(beta D)); 2^-46 is the guard */
  const double eps = 0x1p-46 * g_guard_scale;
  int certain = 1;
  if (k < K && !((double)(W[k] - Ws) >= tau * (1.0 + eps))) certain = 0;
  if (k - 1 > s && !((double)(W[k - 1] - Ws) < tau * (1.0 - eps))) certain = 0;
  if (certain) return k;
  ++*guard;
  const hp_t tau_h = ldexpl(-logl((hp_t)up) / ((hp_t)c->beta * (hp_t)c->p.D), 58);
  lo = s + 1;
  hi = K;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if ((hp_t)(W[mid] - Ws) >= tau_h) hi = mid; else lo = mid + 1;
  }
  return lo;
}

/* Candidate survives iff u q_k < 1 - P_ij, q_k = 1 - exp(-2 beta Vmax), P_ij of Eq. (2). */
static int survives(const sco_ref_ctx* c, const double Si[3], const double Sj[3], int32_t dx,
                    int32_t dy, int64_t r2, uint64_t A, double cc, uint64_t wU, int64_t* guard) {
  const double D = c->p.D, beta = c->beta;
  const double u1 = unif(wU);
  const double Vm = (D * (double)A) * 0x1p-59;
  const double V = ref_V(D, cc, r2, Si, Sj, dx, dy);
  const double b = beta * (V - Vm);
  const double a = (2.0 * beta) * Vm;
  const double pr = -expm1(b);
  const double q = -expm1(-a);
  const double mu = pr - u1 * q;
  const double dV = 0x1p-47 * D * cc * (double)r2;
  const double B = g_guard_scale *
      2.0 * (beta * (dV + 0x1p-52 * Vm) + 0x1p-52 * fabs(b) + 0x1p-49 * (fabs(pr) + q));
  if (mu > B) return 1;
  if (mu < -B) return 0;
  ++*guard;
  const hp_t Vh = ref_V_hp(D, cc, r2, Si, Sj, dx, dy);
  const hp_t Vmh = ldexpl((hp_t)D * (hp_t)A, -59);
  const hp_t bh = (hp_t)beta * (Vh - Vmh);
  const hp_t ah = 2.0L * (hp_t)beta * Vmh;
  return (hp_t)u1 * (-expm1l(-ah)) < -expm1l(bh);
}

typedef struct {
  int32_t *i, *j, *m, *f;
  int64_t n, cap;
} ebuf_t;

static int ebuf_push(ebuf_t* b, int32_t i, int32_t j, int32_t m, int32_t f) {
  if (b->n == b->cap) {
    int64_t nc = b->cap ? 2 * b->cap : 1024;
    int32_t* ni = (int32_t*)realloc(b->i, nc * sizeof(int32_t));
    if (ni) b->i = ni;
    int32_t* nj = (int32_t*)realloc(b->j, nc * sizeof(int32_t));
    if (nj) b->j = nj;
    int32_t* nm = (int32_t*)realloc(b->m, nc * sizeof(int32_t));
    if (nm) b->m = nm;
    int32_t* nf = (int32_t*)realloc(b->f, nc * sizeof(int32_t));
    if (nf) b->f = nf;
    if (!ni || !nj || !nm || !nf) return SCO_REF_ENOMEM;
    b->cap = nc;
  }
  b->i[b->n] = i;
  b->j[b->n] = j;
  b->m[b->n] = m;
  b->f[b->n] = f;
  b->n++;
  return SCO_REF_OK;
}

/* Switch every pair at epoch e (uniforms: Philox tag SWITCH, counter (i, e, n/2), draw n
 * uses words 2(n%2) for the exponential and 2(n%2)+1 for the survival test). */
static int do_switch(sco_ref_ctx* c, uint32_t e) {
  const int64_t N = c->N;
  const int32_t Lx = c->p.Lx, Ly = c->p.Ly;
  const int has_J = c->p.J != 0.0;
  int nt = 1;
#ifdef _OPENMP
  nt = omp_get_max_threads();
#endif
  ebuf_t* bufs = (ebuf_t*)calloc(nt, sizeof(ebuf_t));
  int64_t* guards = (int64_t*)calloc(nt, sizeof(int64_t));
  int* errs = (int*)calloc(nt, sizeof(int));
  if (!bufs || !guards || !errs) {
    free(bufs); free(guards); free(errs);
    return SCO_REF_ENOMEM;
  }
#pragma omp parallel num_threads(nt)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    int64_t lo_i = N * tid / nt, hi_i = N * (tid + 1) / nt;
    ebuf_t* b = &bufs[tid];
    for (int64_t i = lo_i; i < hi_i; ++i) {
      const int32_t x = (int32_t)(i % Lx), y = (int32_t)(i / Lx);
      double Si[3];
      spin_get(c, i, Si);
      const int64_t first = b->n;
      int64_t s = -1;
      uint64_t w[4];
      for (uint64_t n = 0;; ++n) {
        if ((n & 1) == 0) draw(c, (uint64_t)i, e, n >> 1, SCO_REF_TAG_SWITCH, w);
        const uint64_t wE = w[2 * (n & 1)], wU = w[2 * (n & 1) + 1];
        const int64_t k = next_candidate(c, s, wE, &guards[tid]);
        if (k >= c->K) break;
        const int32_t xj = x + c->tdx[k], yj = y + c->tdy[k];
        if (xj >= 0 && xj < Lx && yj < Ly) {
          const int64_t j = xj + (int64_t)Lx * yj;
          double Sj[3];
          spin_get(c, j, Sj);
          if (survives(c, Si, Sj, c->tdx[k], c->tdy[k], c->tr2[k], c->tA[k], c->tc[k], wU,
                       &guards[tid]))
            errs[tid] |= ebuf_push(b, (int32_t)i, (int32_t)j, (int32_t)k, 1);
        }
        s = k;
      }
      if (has_J) {
        /* nearest-neighbour exchange bonds join the colouring graph (Sec. 3.1 applies the
         * switching to the dipolar term only; same-colour spins must not share a bond) */
        for (int q = 0; q < 2; ++q) {
          const int64_t mq = c->m_nn[q];
          if (mq < 0) continue;
          const int32_t xj = x + c->tdx[mq], yj = y + c->tdy[mq];
          if (xj >= Lx || yj >= Ly) continue;
          int64_t pos = first;
          while (pos < b->n && b->m[pos] < mq) ++pos;
          if (pos < b->n && b->m[pos] == mq) {
            b->f[pos] |= 2;
            continue;
          }
          errs[tid] |= ebuf_push(b, 0, 0, 0, 0);
          for (int64_t r = b->n - 1; r > pos; --r) {
            b->i[r] = b->i[r - 1]; b->j[r] = b->j[r - 1];
            b->m[r] = b->m[r - 1]; b->f[r] = b->f[r - 1];
          }
          b->i[pos] = (int32_t)i;
          b->j[pos] = (int32_t)(xj + (int64_t)Lx * yj);
          b->m[pos] = (int32_t)mq;
          b->f[pos] = 2;
        }
      }
    }
  }
  int err = 0;
  int64_t total = 0;
  for (int t = 0; t < nt; ++t) {
    err |= errs[t];
    total += bufs[t].n;
    c->guard_hits += guards[t];
  }
  free_graph(c);
  if (!err) {
    int64_t cap = total > 0 ? total : 1;
    c->ei = (int32_t*)malloc(cap * sizeof(int32_t));
    c->ej = (int32_t*)malloc(cap * sizeof(int32_t));
    c->em = (int32_t*)malloc(cap * sizeof(int32_t));
    c->ef = (int32_t*)malloc(cap * sizeof(int32_t));
    if (!c->ei || !c->ej || !c->em || !c->ef) err = SCO_REF_ENOMEM;
  }
  if (!err) {
    int64_t o = 0;
    for (int t = 0; t < nt; ++t) {
      memcpy(c->ei + o, bufs[t].i, bufs[t].n * sizeof(int32_t));
      memcpy(c->ej + o, bufs[t].j, bufs[t].n * sizeof(int32_t));
      memcpy(c->em + o, bufs[t].m, bufs[t].n * sizeof(int32_t));
      memcpy(c->ef + o, bufs[t].f, bufs[t].n * sizeof(int32_t));
      o += bufs[t].n;
    }
    c->ne = total;
  }
  for (int t = 0; t < nt; ++t) {
    free(bufs[t].i); free(bufs[t].j); free(bufs[t].m); free(bufs[t].f);
  }
  free(bufs); free(guards); free(errs);
  if (err) return err;

  /* symmetric CSR; each row sorted by neighbour index */
  c->row_ptr = (int64_t*)calloc(N + 1, sizeof(int64_t));
  c->nnz = 2 * c->ne;
  c->col = (uint32_t*)malloc((c->nnz > 0 ? c->nnz : 1) * sizeof(uint32_t));
  int64_t* cur = (int64_t*)malloc((N + 1) * sizeof(int64_t));
  if (!c->row_ptr || !c->col || !cur) {
    free(cur);
    return SCO_REF_ENOMEM;
  }
  for (int64_t q = 0; q < c->ne; ++q) {
    c->row_ptr[c->ei[q] + 1]++;
    c->row_ptr[c->ej[q] + 1]++;
  }
  for (int64_t i = 0; i < N; ++i) c->row_ptr[i + 1] += c->row_ptr[i];
  memcpy(cur, c->row_ptr, (N + 1) * sizeof(int64_t));
  for (int64_t q = 0; q < c->ne; ++q) {
    const uint32_t flag = (c->ef[q] & 1) ? 0u : SCO_REF_EXCH_ONLY;
    c->col[cur[c->ei[q]]++] = (uint32_t)c->ej[q] | flag;
    c->col[cur[c->ej[q]]++] = (uint32_t)c->ei[q] | flag;
  }
  free(cur);
  c->max_degree = 0;
  c->max_degree_dip = 0;
  for (int64_t i = 0; i < N; ++i) {
    uint32_t* r = c->col + c->row_ptr[i];
    const int64_t n = c->row_ptr[i + 1] - c->row_ptr[i];
    for (int64_t a = 1; a < n; ++a) { /* insertion sort by neighbour index */
      uint32_t v = r[a];
      int64_t b = a - 1;
      while (b >= 0 && (r[b] & 0x7FFFFFFFu) > (v & 0x7FFFFFFFu)) {
        r[b + 1] = r[b];
        --b;
      }
      r[b + 1] = v;
    }
    int32_t nd = 0;
    for (int64_t a = 0; a < n; ++a) nd += (r[a] & SCO_REF_EXCH_ONLY) ? 0 : 1;
    if (n > c->max_degree) c->max_degree = (int32_t)n;
    if (nd > c->max_degree_dip) c->max_degree_dip = nd;
  }
  c->graph_epoch = e;
  c->colour_valid = 0;
  return SCO_REF_OK;
}

int sco_ref_switch(sco_ref_ctx* c) {
  if (!c) return SCO_REF_EINVAL;
  return do_switch(c, (uint32_t)(c->t / c->p.n_sw));
}

int sco_ref_switch_epoch(sco_ref_ctx* c, uint32_t epoch) {
  if (!c) return SCO_REF_EINVAL;
  return do_switch(c, epoch);
}

/* ---- step (2) of Fig. 1: Kuhn-Wattenhofer colouring -------------------------------- */
/* Sec. 2.3.3.  Vertex v starts with colour v; with g = Delta + 1 the level-0 group of v
 * is floor(v / g) and its colour inside the group is v mod g.  At level p = 1..M, with
 * M = ceil(log2 ceil(N / g)), neighbouring groups merge pairwise (group index >> p) and
 * the colours of the right half are shifted to [g, 2g).  Colour reduction inside every
 * merged group then runs in synchronous rounds until every colour is <= Delta:
 *   variant 0, step (2)' of Sec. 2.3.2: a vertex whose colour is > Delta and larger
 *              than the colour of every neighbour in its group takes the smallest colour
 *              in [0, Delta] that no neighbour in its group holds;
 *   variant 1, step (2) of Sec. 2.3.2: in round alpha = 2g-1, ..., g the vertices with
 *              colour alpha do the same.
 * Readings: groups whose size is not a power of two times g are simply shorter (the
 * last group) or empty; the palette choice is the smallest free colour; "locally
 * maximum" is strict. */
static int kw_same_group(int64_t u, int64_t v, int64_t g, int p) { return (u / g) >> p == (v / g) >> p; }

static int kw_local_max(int64_t v, const int64_t* rp, const uint32_t* col, const int32_t* lc,
                        int64_t g, int p) {
  for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
    const int64_t u = col[e] & 0x7FFFFFFFu;
    if (kw_same_group(u, v, g, p) && lc[u] >= lc[v]) return 0;
  }
  return 1;
}

static int32_t kw_smallest_free(int64_t v, const int64_t* rp, const uint32_t* col,
                                const int32_t* lc, int64_t g, int p, uint8_t* mark) {
  memset(mark, 0, (size_t)g);
  for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
    const int64_t u = col[e] & 0x7FFFFFFFu;
    if (kw_same_group(u, v, g, p) && lc[u] < g) mark[lc[u]] = 1;
  }
  for (int64_t q = 0; q < g; ++q)
    if (!mark[q]) return (int32_t)q;
  return -1; /* impossible: v has at most Delta = g - 1 neighbours */
}

int sco_ref_kw_colour_graph(int64_t N, const int64_t* rp, const uint32_t* col, int32_t variant,
                            int32_t* colour, int32_t* rounds, int32_t* max_degree) {
  if (N < 0 || (N > 0 && (!rp || !colour)) || variant < 0 || variant > 1) return SCO_REF_EINVAL;
  int64_t delta = 0;
  for (int64_t i = 0; i < N; ++i)
    if (rp[i + 1] - rp[i] > delta) delta = rp[i + 1] - rp[i];
  const int64_t g = delta + 1;
  const int64_t G = N > 0 ? (N + g - 1) / g : 0;
  int M = 0;
  while (((int64_t)1 << M) < G) ++M;
  int32_t* lc = colour;
  for (int64_t i = 0; i < N; ++i) lc[i] = (int32_t)(i % g);
  int64_t* pend = (int64_t*)malloc((N > 0 ? N : 1) * sizeof(int64_t));
  int32_t* dec = (int32_t*)malloc((N > 0 ? N : 1) * sizeof(int32_t));
  if (!pend || !dec) {
    free(pend); free(dec);
    return SCO_REF_ENOMEM;
  }
  int32_t t_r = 0;
  int nt = 1;
#ifdef _OPENMP
  nt = omp_get_max_threads();
#endif
  uint8_t* marks = (uint8_t*)malloc((size_t)nt * (size_t)g);
  if (!marks) {
    free(pend); free(dec);
    return SCO_REF_ENOMEM;
  }
  for (int p = 1; p <= M; ++p) {
    int64_t np = 0;
    for (int64_t i = 0; i < N; ++i) {
      if (((i / g) >> (p - 1)) & 1) {
        lc[i] += (int32_t)g;
        pend[np++] = i;
      }
    }
    if (variant == 0) {
      while (np > 0) {
        ++t_r;
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < np; ++q) {
          int tid = 0;
#ifdef _OPENMP
          tid = omp_get_thread_num();
#endif
          const int64_t v = pend[q];
          dec[q] = kw_local_max(v, rp, col, lc, g, p)
                       ? kw_smallest_free(v, rp, col, lc, g, p, marks + (size_t)tid * g)
                       : -1;
        }
        int64_t keep = 0;
        for (int64_t q = 0; q < np; ++q) {
          if (dec[q] >= 0) lc[pend[q]] = dec[q];
          else pend[keep++] = pend[q];
        }
        np = keep;
      }
    } else {
      for (int64_t alpha = 2 * g - 1; alpha >= g; --alpha) {
        ++t_r;
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < np; ++q) {
          int tid = 0;
#ifdef _OPENMP
          tid = omp_get_thread_num();
#endif
          const int64_t v = pend[q];
          dec[q] = lc[v] == alpha ? kw_smallest_free(v, rp, col, lc, g, p, marks + (size_t)tid * g)
                                  : -1;
        }
        for (int64_t q = 0; q < np; ++q)
          if (dec[q] >= 0) lc[pend[q]] = dec[q];
      }
    }
  }
  free(pend); free(dec); free(marks);
  if (rounds) *rounds = t_r;
  if (max_degree) *max_degree = (int32_t)delta;
  return SCO_REF_OK;
}

int sco_ref_colour(sco_ref_ctx* c, int32_t* n_colours) {
  if (!c) return SCO_REF_EINVAL;
  if (c->graph_epoch < 0) {
    int st = sco_ref_switch(c);
    if (st) return st;
  }
  int32_t rounds = 0, delta = 0;
  int st = sco_ref_kw_colour_graph(c->N, c->row_ptr, c->col, c->p.colour_variant, c->colour,
                                   &rounds, &delta);
  if (st) return st;
  c->kw_rounds = rounds;
  c->g = delta + 1;
  /* colour classes: sites sorted by (colour, index) (Fig. 1 step (3)) */
  free(c->off);
  c->off = (int64_t*)calloc((size_t)c->g + 1, sizeof(int64_t));
  if (!c->off) return SCO_REF_ENOMEM;
  for (int64_t i = 0; i < c->N; ++i) c->off[c->colour[i] + 1]++;
  for (int32_t q = 0; q < c->g; ++q) c->off[q + 1] += c->off[q];
  int64_t* cur = (int64_t*)malloc(((size_t)c->g + 1) * sizeof(int64_t));
  if (!cur) return SCO_REF_ENOMEM;
  memcpy(cur, c->off, ((size_t)c->g + 1) * sizeof(int64_t));
  for (int64_t i = 0; i < c->N; ++i) c->perm[cur[c->colour[i]]++] = i;
  free(cur);
  c->colour_valid = 1;
  if (n_colours) {
    int32_t nc = 0;
    for (int32_t q = 0; q < c->g; ++q) nc += c->off[q + 1] > c->off[q];
    *n_colours = nc;
  }
  return SCO_REF_OK;
}

/* ---- step (B): colour-class Metropolis ---------------------------------------------- */
/* Accept iff u < exp(-beta dE'), i.e. u == 0 or ln u + beta dE' < 0, where
 * beta dE' = sum over surviving pairs of beta [Vbar(S') - Vbar(S)] - beta J (S'-S).h_NN
 * and beta Vbar = beta V - log(1 - exp(beta (V - Vmax))) (Eq. (3)). */
static int accept_move(const sco_ref_ctx* c, int64_t i, const double S[3], const double Sn[3],
                       double u, int64_t* guard) {
  if (u == 0.0) return 1;
  const double D = c->p.D, beta = c->beta, J = c->p.J;
  const int32_t Lx = c->p.Lx, Ly = c->p.Ly;
  const int32_t xi = (int32_t)(i % Lx), yi = (int32_t)(i / Lx);
  double sum = 0.0, sumabs = 0.0, bnd = 0.0;
  int64_t nterm = 0;
  int fp64_ok = 1;
  for (int64_t e = c->row_ptr[i]; e < c->row_ptr[i + 1]; ++e) {
    if (c->col[e] & SCO_REF_EXCH_ONLY) continue;
    const int64_t j = c->col[e];
    const int32_t dx = (int32_t)(j % Lx) - xi, dy = (int32_t)(j / Lx) - yi;
    const int64_t r2 = (int64_t)dx * dx + (int64_t)dy * dy;
    const double cc = ref_coupling_c(r2);
    const double Vm = (D * (double)ref_hazard_A(r2)) * 0x1p-59;
    double Sj[3];
    spin_get(c, j, Sj);
    const double Vn = ref_V(D, cc, r2, Sn, Sj, dx, dy);
    const double Vo = ref_V(D, cc, r2, S, Sj, dx, dy);
    const double xn = beta * (Vn - Vm), xo = beta * (Vo - Vm);
    if (!(xn < 0.0) || !(xo < 0.0)) {
      fp64_ok = 0;
      break;
    }
    double sn, so;
    const double Ln = ref_log1mexp(xn, &sn), Lo = ref_log1mexp(xo, &so);
    const double dbv = beta * (Vn - Vo);
    const double term = (dbv - Ln) + Lo;
    sum += term;
    sumabs += fabs(term);
    ++nterm;
    const double dV = 0x1p-47 * D * cc * (double)r2;
    const double dxn = beta * (dV + 0x1p-52 * Vm) + 0x1p-52 * fabs(xn);
    const double dxo = beta * (dV + 0x1p-52 * Vm) + 0x1p-52 * fabs(xo);
    if (dxn > 0.25 * fabs(xn) || dxo > 0.25 * fabs(xo)) {
      /* the first-order bound below needs |dx| well inside |x| */
      fp64_ok = 0;
      break;
    }
    bnd += 2.0 * beta * dV + 0x1p-51 * fabs(dbv) + sn * dxn + so * dxo +
           0x1p-49 * (2.0 + fabs(Ln) + fabs(Lo)) + 0x1p-51 * (fabs(dbv) + fabs(Ln) + fabs(Lo));
  }
  if (fp64_ok && J != 0.0) {
    double h[3] = {0.0, 0.0, 0.0};
    const int64_t nb[4] = {xi > 0 ? i - 1 : -1, xi + 1 < Lx ? i + 1 : -1, yi > 0 ? i - Lx : -1,
                           yi + 1 < Ly ? i + Lx : -1};
    for (int q = 0; q < 4; ++q) {
      if (nb[q] < 0) continue;
      double Sj[3];
      spin_get(c, nb[q], Sj);
      h[0] += Sj[0]; h[1] += Sj[1]; h[2] += Sj[2];
    }
    const double dot = (Sn[0] - S[0]) * h[0] + (Sn[1] - S[1]) * h[1] + (Sn[2] - S[2]) * h[2];
    const double tex = -(beta * J) * dot;
    sum += tex;
    sumabs += fabs(tex);
    ++nterm;
    bnd += 0x1p-44 * fabs(beta * J);
  }
  if (fp64_ok) {
    const double lu = log(u);
    const double mu = lu + sum;
    const double B = g_guard_scale * 2.0 *
                     (bnd + (double)(nterm + 1) * 0x1p-52 * sumabs + 0x1p-50 * fabs(lu) +
                      0x1p-52 * fabs(mu));
    if (mu < -B) return 1;
    if (mu > B) return 0;
  }
  ++*guard;
  /* extended precision re-evaluation of the same real comparison */
  hp_t sh = 0.0L;
  for (int64_t e = c->row_ptr[i]; e < c->row_ptr[i + 1]; ++e) {
    if (c->col[e] & SCO_REF_EXCH_ONLY) continue;
    const int64_t j = c->col[e];
    const int32_t dx = (int32_t)(j % Lx) - xi, dy = (int32_t)(j / Lx) - yi;
    const int64_t r2 = (int64_t)dx * dx + (int64_t)dy * dy;
    const double cc = ref_coupling_c(r2);
    const hp_t Vm = ldexpl((hp_t)D * (hp_t)ref_hazard_A(r2), -59);
    double Sj[3];
    spin_get(c, j, Sj);
    const hp_t Vn = ref_V_hp(D, cc, r2, Sn, Sj, dx, dy);
    const hp_t Vo = ref_V_hp(D, cc, r2, S, Sj, dx, dy);
    const hp_t xn = (hp_t)beta * (Vn - Vm), xo = (hp_t)beta * (Vo - Vm);
    if (!(xn < 0.0L)) return 0; /* pseudointeraction +inf: reject */
    sh += (hp_t)beta * (Vn - Vo) - ref_log1mexp_hp(xn) + ref_log1mexp_hp(xo);
  }
  if (J != 0.0) {
    hp_t h[3] = {0.0L, 0.0L, 0.0L};
    const int64_t nb[4] = {xi > 0 ? i - 1 : -1, xi + 1 < Lx ? i + 1 : -1, yi > 0 ? i - Lx : -1,
                           yi + 1 < Ly ? i + Lx : -1};
    for (int q = 0; q < 4; ++q) {
      if (nb[q] < 0) continue;
      double Sj[3];
      spin_get(c, nb[q], Sj);
      h[0] += Sj[0]; h[1] += Sj[1]; h[2] += Sj[2];
    }
    const hp_t dot = ((hp_t)Sn[0] - S[0]) * h[0] + ((hp_t)Sn[1] - S[1]) * h[1] +
                     ((hp_t)Sn[2] - S[2]) * h[2];
    sh += -((hp_t)beta * (hp_t)J) * dot;
  }
  return logl((hp_t)u) + sh < 0.0L;
}

/* One MC step t: colours in ascending order; inside a colour every site is independent
 * (no surviving pair or exchange bond joins two sites of one colour, Sec. 2.2), so the
 * order inside a class does not matter.  Proposal: Philox tag PROPOSE, counter
 * (i, t, a); attempt a uses words 0, 1 (Marsaglia) and the acceptance uniform is
 * word 2 of the successful attempt.  64 failed attempts leave the spin unchanged. */
static void mc_step(sco_ref_ctx* c) {
  const int64_t N = c->N;
  const uint64_t t = (uint64_t)c->t;
  int64_t guard = 0;
  for (int32_t q = 0; q < c->g; ++q) {
#pragma omp parallel for schedule(static) reduction(+ : guard)
    for (int64_t idx = c->off[q]; idx < c->off[q + 1]; ++idx) {
      const int64_t i = c->perm[idx];
      double S[3], Sn[3];
      spin_get(c, i, S);
      int found = 0;
      double u = 0.0;
      for (uint64_t a = 0; a < 64; ++a) {
        uint64_t w[4];
        draw(c, (uint64_t)i, t, a, SCO_REF_TAG_PROPOSE, w);
        if (sco_ref_marsaglia(w[0], w[1], Sn)) {
          u = unif(w[2]);
          found = 1;
          break;
        }
      }
      int ok = 0;
      if (found) ok = accept_move(c, i, S, Sn, u, &guard);
      if (ok) {
        c->s[i] = Sn[0];
        c->s[N + i] = Sn[1];
        c->s[2 * N + i] = Sn[2];
      }
      c->acc[i] = (uint8_t)ok;
    }
  }
  c->guard_hits += guard;
}

int sco_ref_sweep(sco_ref_ctx* c, int32_t n_mcs) {
  if (!c || n_mcs < 0) return SCO_REF_EINVAL;
  for (int32_t k = 0; k < n_mcs; ++k) {
    const int64_t e = c->t / c->p.n_sw;
    if (c->graph_epoch != e) {
      int st = do_switch(c, (uint32_t)e);
      if (st) return st;
    }
    if (!c->colour_valid) {
      int st = sco_ref_colour(c, NULL);
      if (st) return st;
    }
    mc_step(c);
    c->t++;
  }
  return SCO_REF_OK;
}

/* ---- observables --------------------------------------------------------------------- */
static hp_t exchange_energy(const sco_ref_params* p, const double* s) {
  const int64_t N = (int64_t)p->Lx * p->Ly;
  hp_t e = 0.0L;
  for (int64_t i = 0; i < N; ++i) {
    const int32_t x = (int32_t)(i % p->Lx), y = (int32_t)(i / p->Lx);
    if (x + 1 < p->Lx)
      e += (hp_t)(s[i] * s[i + 1] + s[N + i] * s[N + i + 1] + s[2 * N + i] * s[2 * N + i + 1]);
    if (y + 1 < p->Ly) {
      const int64_t j = i + p->Lx;
      e += (hp_t)(s[i] * s[j] + s[N + i] * s[N + j] + s[2 * N + i] * s[2 * N + j]);
    }
  }
  return -(hp_t)p->J * e;
}

int sco_ref_observables(sco_ref_ctx* c, sco_ref_obs* o, int32_t want_full) {
  if (!c || !o) return SCO_REF_EINVAL;
  memset(o, 0, sizeof(*o));
  const int64_t N = c->N;
  const int32_t Lx = c->p.Lx, Ly = c->p.Ly;
  const hp_t eex = exchange_energy(&c->p, c->s);
  hp_t ep = 0.0L;
  int64_t ndip = 0;
  if (c->graph_epoch >= 0) {
    for (int64_t q = 0; q < c->ne; ++q) {
      if (!(c->ef[q] & 1)) continue;
      ++ndip;
      const int64_t i = c->ei[q], j = c->ej[q];
      const int32_t dx = (int32_t)(j % Lx) - (int32_t)(i % Lx);
      const int32_t dy = (int32_t)(j / Lx) - (int32_t)(i / Lx);
      const int64_t r2 = (int64_t)dx * dx + (int64_t)dy * dy;
      double Si[3], Sj[3];
      spin_get(c, i, Si);
      spin_get(c, j, Sj);
      const double V = ref_V(c->p.D, ref_coupling_c(r2), r2, Si, Sj, dx, dy);
      ep += (hp_t)sco_ref_pseudo(c->beta, V, sco_ref_vmax(c->p.D, r2));
    }
  }
  o->e_exchange = (double)eex;
  o->e_switched = (double)(ep + eex);
  o->e_full = want_full ? sco_ref_full_energy(&c->p, c->s) : NAN;
  hp_t mx = 0, my = 0, mz = 0, mphi = 0;
  const double rcx = 0.5 * (Lx - 1), rcy = 0.5 * (Ly - 1);
  for (int64_t i = 0; i < N; ++i) {
    mx += c->s[i];
    my += c->s[N + i];
    mz += c->s[2 * N + i];
    const double ux = (double)(i % Lx) - rcx, uy = (double)(i / Lx) - rcy;
    const double nr = sqrt(ux * ux + uy * uy);
    if (nr > 0.0) mphi += (hp_t)((c->s[i] * uy - c->s[N + i] * ux) / nr);
  }
  o->mx = (double)(mx / N);
  o->my = (double)(my / N);
  o->mz = (double)(mz / N);
  o->m_abs = sqrt(o->mx * o->mx + o->my * o->my + o->mz * o->mz);
  o->m_phi = (double)(mphi / N);
  o->n_edges = ndip;
  o->max_degree = c->graph_epoch >= 0 ? c->max_degree : 0;
  o->max_degree_dipolar = c->graph_epoch >= 0 ? c->max_degree_dip : 0;
  o->kw_rounds = c->colour_valid ? c->kw_rounds : 0;
  int32_t nc = 0;
  if (c->colour_valid)
    for (int32_t q = 0; q < c->g; ++q) nc += c->off[q + 1] > c->off[q];
  o->n_colours = nc;
  o->sweeps_done = c->t;
  o->guard_hits = c->guard_hits;
  return SCO_REF_OK;
}

/* ---- accessors ------------------------------------------------------------------------ */
int64_t sco_ref_n_sites(const sco_ref_ctx* c) { return c ? c->N : 0; }
int64_t sco_ref_n_entries(const sco_ref_ctx* c) { return c ? c->nnz : 0; }
int64_t sco_ref_n_half_edges(const sco_ref_ctx* c) { return c ? c->ne : 0; }
int64_t sco_ref_sweeps_done(const sco_ref_ctx* c) { return c ? c->t : 0; }

int sco_ref_get_spins(const sco_ref_ctx* c, double* xyz) {
  if (!c || !xyz) return SCO_REF_EINVAL;
  memcpy(xyz, c->s, 3 * c->N * sizeof(double));
  return SCO_REF_OK;
}

int sco_ref_set_spins(sco_ref_ctx* c, const double* xyz) {
  if (!c || !xyz) return SCO_REF_EINVAL;
  memcpy(c->s, xyz, 3 * c->N * sizeof(double));
  return SCO_REF_OK;
}

int sco_ref_get_graph(const sco_ref_ctx* c, int64_t* row_ptr, uint32_t* col, int32_t* colour) {
  if (!c) return SCO_REF_EINVAL;
  if ((row_ptr || col) && c->graph_epoch < 0) return SCO_REF_EINVAL;
  if (colour && !c->colour_valid) return SCO_REF_EINVAL;
  if (row_ptr) memcpy(row_ptr, c->row_ptr, (c->N + 1) * sizeof(int64_t));
  if (col && c->nnz) memcpy(col, c->col, c->nnz * sizeof(uint32_t));
  if (colour) memcpy(colour, c->colour, c->N * sizeof(int32_t));
  return SCO_REF_OK;
}

int sco_ref_get_edges(const sco_ref_ctx* c, int64_t* i, int64_t* j, int64_t* m, int32_t* f) {
  if (!c || c->graph_epoch < 0) return SCO_REF_EINVAL;
  for (int64_t q = 0; q < c->ne; ++q) {
    if (i) i[q] = c->ei[q];
    if (j) j[q] = c->ej[q];
    if (m) m[q] = c->em[q];
    if (f) f[q] = c->ef[q];
  }
  return SCO_REF_OK;
}

int sco_ref_get_classes(const sco_ref_ctx* c, int64_t* perm, int64_t* off) {
  if (!c || !c->colour_valid) return SCO_REF_EINVAL;
  if (perm) memcpy(perm, c->perm, c->N * sizeof(int64_t));
  if (off) memcpy(off, c->off, ((size_t)c->g + 1) * sizeof(int64_t));
  return SCO_REF_OK;
}

int sco_ref_get_accepts(const sco_ref_ctx* c, uint8_t* acc) {
  if (!c || !acc) return SCO_REF_EINVAL;
  memcpy(acc, c->acc, c->N);
  return SCO_REF_OK;
}

int sco_ref_get_params_(const sco_ref_ctx* c, sco_ref_params* p) {
  if (!c || !p) return SCO_REF_EINVAL;
  *p = c->p;
  return SCO_REF_OK;
}

/* Run n MC steps and record, after each, the full energy per spin (Eq. (6), direct sum) and
 * |m|; used by the equilibrium checks against the plain Metropolis sampler. */
int sco_ref_run_series(sco_ref_ctx* c, int64_t n_mcs, double* e_per_spin, double* m_abs) {
  if (!c || n_mcs < 0) return SCO_REF_EINVAL;
  for (int64_t k = 0; k < n_mcs; ++k) {
    int st = sco_ref_sweep(c, 1);
    if (st) return st;
    if (e_per_spin) e_per_spin[k] = sco_ref_full_energy(&c->p, c->s) / (double)c->N;
    if (m_abs) {
      double m[3] = {0, 0, 0};
      for (int64_t i = 0; i < c->N; ++i) {
        m[0] += c->s[i];
        m[1] += c->s[c->N + i];
        m[2] += c->s[2 * c->N + i];
      }
      m_abs[k] = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / (double)c->N;
    }
  }
  return SCO_REF_OK;
}

/* ---- temperature (the cooling protocol of Sec. 3.1) ------------------------------------ */
int sco_ref_set_temperature(sco_ref_ctx* c, double T) {
  if (!c || !(T > 0.0) || !isfinite(T)) return SCO_REF_EINVAL;
  c->p.T = T;
  c->beta = 1.0 / T;
  c->bD = c->beta * c->p.D;
  /* the switched graph belongs to the old temperature: switch (and colour) again before the
     next MC step, at the same epoch number */
  c->graph_epoch = -1;
  c->colour_valid = 0;
  return SCO_REF_OK;
}

/* ---- graph diagnostics (Sec. 3.2, Figs. 5 and 6; Sec. 3.3, Eq. (9)) -------------------- */
/* floor(sqrt(r2)) exactly: the rounded root corrected by integer comparisons */
static int64_t floor_sqrt(int64_t r2) {
  int64_t s = (int64_t)sqrt((double)r2);
  while (s * s > r2) --s;
  while ((s + 1) * (s + 1) <= r2) ++s;
  return s;
}

/* distance shell of a pair: bin b holds b + 1 <= r < b + 2, the last bin everything beyond */
static int32_t shell_bin(int64_t r2, int32_t n_rbins) {
  const int64_t b = floor_sqrt(r2) - 1;
  return (int32_t)(b < n_rbins - 1 ? b : n_rbins - 1);
}

/* cell of site (x, y) in a cells_x x cells_y split of the lattice into rectangles */
static int64_t cell_of(const sco_ref_params* p, int64_t i, int32_t cx, int32_t cy) {
  const int64_t x = i % p->Lx, y = i / p->Lx;
  return (x * cx) / p->Lx + (int64_t)cx * ((y * cy) / p->Ly);
}

int sco_ref_graph_stats(const sco_ref_ctx* c, int32_t cells_x, int32_t cells_y, int32_t n_rbins,
                        sco_ref_gstats* out, int64_t* survived, int64_t* pairs,
                        double* p_survive, double* delta_r) {
  if (!c || !out || cells_x < 1 || cells_y < 1 || cells_x > c->p.Lx || cells_y > c->p.Ly ||
      n_rbins < 1)
    return SCO_REF_EINVAL;
  if (c->graph_epoch < 0 || !c->colour_valid) return SCO_REF_EINVAL;
  const int32_t Lx = c->p.Lx, Ly = c->p.Ly;
  const int64_t ncell = (int64_t)cells_x * cells_y;
  int64_t* surv = (int64_t*)calloc((size_t)n_rbins, sizeof(int64_t));
  int64_t* npair = (int64_t*)calloc((size_t)n_rbins, sizeof(int64_t));
  int64_t* K = (int64_t*)calloc((size_t)(ncell * c->g), sizeof(int64_t));
  if (!surv || !npair || !K) {
    free(surv);
    free(npair);
    free(K);
    return SCO_REF_ENOMEM;
  }
  /* every pair of the open lattice once: displacement d of the half plane, (Lx-|dx|)(Ly-|dy|)
     site pairs (i, i + d) inside the lattice */
  for (int64_t m = 0; m < c->K; ++m) {
    const int64_t ax = c->tdx[m] < 0 ? -c->tdx[m] : c->tdx[m];
    const int64_t ay = c->tdy[m];
    npair[shell_bin(c->tr2[m], n_rbins)] += (Lx - ax) * (Ly - ay);
  }
  /* surviving dipolar pairs by shell, and those whose sites lie in different cells (P_IPC) */
  int64_t ndip = 0, ncross = 0;
  for (int64_t q = 0; q < c->ne; ++q) {
    if (!(c->ef[q] & 1)) continue;
    const int64_t i = c->ei[q], j = c->ej[q];
    const int64_t dx = j % Lx - i % Lx, dy = j / Lx - i / Lx;
    ++surv[shell_bin(dx * dx + dy * dy, n_rbins)];
    ++ndip;
    if (cell_of(&c->p, i, cells_x, cells_y) != cell_of(&c->p, j, cells_x, cells_y)) ++ncross;
  }
  /* sites of each colour in each cell; Eq. (9) per colour: (K_max - K_ave) / K_ave with K_ave
     the class size over the number of cells */
  for (int64_t i = 0; i < c->N; ++i)
    ++K[(int64_t)c->colour[i] * ncell + cell_of(&c->p, i, cells_x, cells_y)];
  double sum = 0.0, dmax = 0.0;
  int32_t nonempty = 0;
  int64_t kmax_sum = 0;
  for (int32_t col = 0; col < c->g; ++col) {
    int64_t tot = 0, kmax = 0;
    for (int64_t q = 0; q < ncell; ++q) {
      const int64_t k = K[(int64_t)col * ncell + q];
      tot += k;
      if (k > kmax) kmax = k;
    }
    kmax_sum += kmax;
    double dr = NAN;
    if (tot > 0) {
      const double kave = (double)tot / (double)ncell;
      dr = ((double)kmax - kave) / kave;
      sum += dr;
      if (dr > dmax) dmax = dr;
      ++nonempty;
    }
    if (delta_r) delta_r[col] = dr;
  }
  for (int32_t b = 0; b < n_rbins; ++b) {
    if (survived) survived[b] = surv[b];
    if (pairs) pairs[b] = npair[b];
    if (p_survive) p_survive[b] = npair[b] > 0 ? (double)surv[b] / (double)npair[b] : NAN;
  }
  out->n_pairs = ndip;
  out->n_cross = ncross;
  out->p_ipc = ndip > 0 ? (double)ncross / (double)ndip : 0.0;
  out->delta_r_mean = nonempty > 0 ? sum / nonempty : 0.0;
  out->delta_r_max = dmax;
  /* each class weighted by its size: the sweep of a colour lasts as long as its fullest cell */
  out->delta_r_weighted = (double)(kmax_sum * ncell) / (double)c->N - 1.0;
  out->n_cells = (int32_t)ncell;
  out->palette = c->g;
  free(surv);
  free(npair);
  free(K);
  return SCO_REF_OK;
}
