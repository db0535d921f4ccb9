/*
 * ref_defn.c -- definitional samplers used to check the oracle's chain
 * statistically.  TEST INFRASTRUCTURE ONLY (see sco_ref.h).
 *
 *  - direct O(N^2) switching: every pair tested on its own (Sec. 2.1 step (A));
 *  - plain single-spin Metropolis on the full Hamiltonian of Eq. (6);
 *  - the full Hamiltonian by direct summation.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "ref_internal.h"

static inline void draw_p(const sco_ref_params* p, uint64_t a0, uint64_t a1, uint64_t a2,
                          uint64_t tag, uint64_t w[4]) {
  uint64_t ctr[4] = {a0, a1, a2, tag};
  uint64_t key[2] = {p->seed, (uint64_t)(uint32_t)p->replica};
  sco_ref_philox(ctr, key, w);
}

/* Accessors into the chain context without exposing its layout. */
int sco_ref_get_params_(const sco_ref_ctx* c, sco_ref_params* p);

int sco_ref_direct_switch(const sco_ref_ctx* c, uint32_t epoch, uint8_t* survive) {
  if (!c || !survive) return SCO_REF_EINVAL;
  sco_ref_params p;
  sco_ref_get_params_(c, &p);
  const int64_t N = (int64_t)p.Lx * p.Ly;
  double* s = (double*)malloc(3 * N * sizeof(double));
  if (!s) return SCO_REF_ENOMEM;
  sco_ref_get_spins(c, s);
  const double beta = 1.0 / p.T;
  memset(survive, 0, (size_t)(N * N));
  for (int64_t i = 0; i < N; ++i) {
    const double Si[3] = {s[i], s[N + i], s[2 * N + i]};
    for (int64_t j = i + 1; j < N; ++j) {
      const double Sj[3] = {s[j], s[N + j], s[2 * N + j]};
      const int32_t dx = (int32_t)(j % p.Lx) - (int32_t)(i % p.Lx);
      const int32_t dy = (int32_t)(j / p.Lx) - (int32_t)(i / p.Lx);
      const int64_t r2 = (int64_t)dx * dx + (int64_t)dy * dy;
      const double V = sco_ref_pair_V(p.D, Si, Sj, dx, dy);
      const double P = sco_ref_switch_prob(beta, V, sco_ref_vmax(p.D, r2));
      uint64_t w[4];
      draw_p(&p, (uint64_t)i, (uint64_t)j, epoch, SCO_REF_TAG_DIRECT, w);
      const double u = (double)(w[0] >> 11) * 0x1p-53;
      survive[i * N + j] = u < 1.0 - P;
    }
  }
  free(s);
  return SCO_REF_OK;
}

/* Local field of site i under H (Eq. (6)): dE for S_i -> S' is (S' - S_i).h_i with
 * h_i = sum_j A_ij S_j, A_ij = D [I/r^3 - 3 r r^T / r^5] - J [j nearest neighbour]. */
static void local_field(const sco_ref_params* p, const double* s, int64_t i, double h[3]) {
  const int64_t N = (int64_t)p->Lx * p->Ly;
  const int32_t xi = (int32_t)(i % p->Lx), yi = (int32_t)(i / p->Lx);
  h[0] = h[1] = h[2] = 0.0;
  for (int64_t j = 0; j < N; ++j) {
    if (j == i) continue;
    const int32_t dx = (int32_t)(j % p->Lx) - xi, dy = (int32_t)(j / p->Lx) - yi;
    const double r2 = (double)dx * dx + (double)dy * dy;
    const double r = sqrt(r2);
    const double ir3 = 1.0 / (r2 * r), ir5 = ir3 / r2;
    const double Sj[3] = {s[j], s[N + j], s[2 * N + j]};
    const double sd = Sj[0] * dx + Sj[1] * dy;
    h[0] += p->D * (Sj[0] * ir3 - 3.0 * dx * sd * ir5);
    h[1] += p->D * (Sj[1] * ir3 - 3.0 * dy * sd * ir5);
    h[2] += p->D * (Sj[2] * ir3);
    if (r2 == 1.0) {
      h[0] -= p->J * Sj[0];
      h[1] -= p->J * Sj[1];
      h[2] -= p->J * Sj[2];
    }
  }
}

double sco_ref_full_energy(const sco_ref_params* p, const double* s) {
  const int64_t N = (int64_t)p->Lx * p->Ly;
  hp_t e = 0.0L;
  for (int64_t i = 0; i < N; ++i) {
    const double Si[3] = {s[i], s[N + i], s[2 * N + i]};
    for (int64_t j = i + 1; j < N; ++j) {
      const double Sj[3] = {s[j], s[N + j], s[2 * N + j]};
      const int32_t dx = (int32_t)(j % p->Lx) - (int32_t)(i % p->Lx);
      const int32_t dy = (int32_t)(j / p->Lx) - (int32_t)(i / p->Lx);
      e += (hp_t)sco_ref_pair_V(p->D, Si, Sj, dx, dy);
      if ((int64_t)dx * dx + (int64_t)dy * dy == 1)
        e -= (hp_t)p->J * (hp_t)(Si[0] * Sj[0] + Si[1] * Sj[1] + Si[2] * Sj[2]);
    }
  }
  return (double)e;
}

int sco_ref_plain_metropolis(const sco_ref_params* p, const double* xyz0, int64_t n_mcs,
                             double* e_per_spin, double* m_abs, double* xyz_out) {
  if (!p || !xyz0 || n_mcs < 0 || p->Lx < 1 || p->Ly < 1 || !(p->T > 0)) return SCO_REF_EINVAL;
  const int64_t N = (int64_t)p->Lx * p->Ly;
  const double beta = 1.0 / p->T;
  double* s = (double*)malloc(3 * N * sizeof(double));
  if (!s) return SCO_REF_ENOMEM;
  memcpy(s, xyz0, 3 * N * sizeof(double));
  double E = sco_ref_full_energy(p, s);
  double M[3] = {0, 0, 0};
  for (int64_t i = 0; i < N; ++i) {
    M[0] += s[i];
    M[1] += s[N + i];
    M[2] += s[2 * N + i];
  }
  for (int64_t t = 0; t < n_mcs; ++t) {
    for (int64_t i = 0; i < N; ++i) {
      double Sn[3];
      uint64_t w[4];
      int found = 0;
      for (uint64_t a = 0; a < 64 && !found; ++a) {
        draw_p(p, (uint64_t)i, (uint64_t)t, a, SCO_REF_TAG_PLAIN, w);
        found = sco_ref_marsaglia(w[0], w[1], Sn);
      }
      if (!found) continue;
      const double u = (double)(w[2] >> 11) * 0x1p-53;
      double h[3];
      local_field(p, s, i, h);
      const double d[3] = {Sn[0] - s[i], Sn[1] - s[N + i], Sn[2] - s[2 * N + i]};
      const double dE = d[0] * h[0] + d[1] * h[1] + d[2] * h[2];
      if (dE <= 0.0 || u < exp(-beta * dE)) {
        s[i] = Sn[0];
        s[N + i] = Sn[1];
        s[2 * N + i] = Sn[2];
        E += dE;
        M[0] += d[0];
        M[1] += d[1];
        M[2] += d[2];
      }
    }
    if (e_per_spin) e_per_spin[t] = E / (double)N;
    if (m_abs) m_abs[t] = sqrt(M[0] * M[0] + M[1] * M[1] + M[2] * M[2]) / (double)N;
  }
  if (xyz_out) memcpy(xyz_out, s, 3 * N * sizeof(double));
  free(s);
  return SCO_REF_OK;
}
