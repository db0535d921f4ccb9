/*
 * ref_model.c -- oracle model: dipolar pair potential, V_max, switching
 * probability, pseudointeraction and the translation-invariant coupling table.
 * TEST INFRASTRUCTURE ONLY (see sco_ref.h).
 */
#include <math.h>
#include <stdlib.h>

#include "ref_internal.h"

double ref_coupling_c(int64_t r2) {
  double q = (double)r2;
  double s = sqrt(q);
  return 1.0 / ((q * q) * s);
}

/* Sec. 2.1: V_max is any constant >= the maximum of V_ij over both spins.
 * For the dipolar pair the maximum of D [S_i.S_j - 3 (S_i.r^)(S_j.r^)] / r^3 over unit
 * spins is 2D/r^3 (largest singular value of (I - 3 r^ r^T), reached at
 * S_i = -S_j = r^).  The oracle takes V_max = D * A * 2^-59 with the integer A
 * below, which exceeds 2^60 / r^3 because the relative rounding of the FP64
 * quotient (< 4 * 2^-53) is smaller than the factor 1 + 2^-50. */
uint64_t ref_hazard_A(int64_t r2) {
  double q = (double)r2;
  double s = sqrt(q);
  double t = 0x1p60 / (q * s);
  double u = t * (1.0 + 0x1p-50);
  return (uint64_t)u + 1u;
}

double sco_ref_vmax(double D, int64_t r2) { return (D * (double)ref_hazard_A(r2)) * 0x1p-59; }

/* Eq. (6), dipolar term of one pair: D [S_i.S_j / r^3 - 3 (S_i.r)(S_j.r) / r^5]
 * = D c(r^2) [r^2 (S_i.S_j) - 3 (S_i.d)(S_j.d)],  c(r^2) ~ r^-5, d = (dx, dy, 0). */
double ref_V(double D, double c, int64_t r2, const double Si[3], const double Sj[3], int32_t dx,
             int32_t dy) {
  double fx = (double)dx, fy = (double)dy;
  double ss = Si[0] * Sj[0] + Si[1] * Sj[1] + Si[2] * Sj[2];
  double pi = Si[0] * fx + Si[1] * fy;
  double pj = Sj[0] * fx + Sj[1] * fy;
  double inner = (double)r2 * ss - 3.0 * (pi * pj);
  return (D * c) * inner;
}

hp_t ref_V_hp(double D, double c, int64_t r2, const double Si[3], const double Sj[3], int32_t dx,
              int32_t dy) {
  hp_t fx = (hp_t)dx, fy = (hp_t)dy;
  hp_t ss = (hp_t)Si[0] * Sj[0] + (hp_t)Si[1] * Sj[1] + (hp_t)Si[2] * Sj[2];
  hp_t pi = (hp_t)Si[0] * fx + (hp_t)Si[1] * fy;
  hp_t pj = (hp_t)Sj[0] * fx + (hp_t)Sj[1] * fy;
  hp_t inner = (hp_t)r2 * ss - 3.0L * (pi * pj);
  return (hp_t)D * (hp_t)c * inner;
}

double sco_ref_pair_V(double D, const double Si[3], const double Sj[3], int32_t dx, int32_t dy) {
  int64_t r2 = (int64_t)dx * dx + (int64_t)dy * dy;
  return ref_V(D, ref_coupling_c(r2), r2, Si, Sj, dx, dy);
}

/* Eq. (2): P_ij = exp[beta (V_ij - V_max)]. */
double sco_ref_switch_prob(double beta, double V, double Vmax) { return exp(beta * (V - Vmax)); }

/* Maechler (2012), "Accurately computing log(1 - exp(-|a|))": log(-expm1(x)) above
 * -ln 2, log1p(-exp(x)) below. */
double ref_log1mexp(double x, double* sens) {
  if (x > -M_LN2) {
    double z = -expm1(x);
    *sens = (1.0 - z) / z;
    return log(z);
  }
  double y = exp(x);
  *sens = 2.0 * y;
  return log1p(-y);
}

hp_t ref_log1mexp_hp(hp_t x) {
  if (x > -logl(2.0L)) return logl(-expm1l(x));
  return log1pl(-expl(x));
}

/* Eq. (3): Vbar_ij = V_ij - beta^-1 log[1 - P_ij]. */
double sco_ref_pseudo(double beta, double V, double Vmax) {
  double sens;
  return V - ref_log1mexp(beta * (V - Vmax), &sens) / beta;
}

/* ---- coupling table ------------------------------------------------------------- */
/* Every unordered pair {i, j} of the open lattice is (i, i + d) for exactly one d of the
 * half plane  {dy > 0, |dx| <= Lx-1, dy <= Ly-1} u {dy = 0, 1 <= dx <= Lx-1}. */
int64_t sco_ref_table_size(int32_t Lx, int32_t Ly) {
  if (Lx < 1 || Ly < 1) return 0;
  return (int64_t)(Lx - 1) + (int64_t)(Ly - 1) * (2 * (int64_t)Lx - 1);
}

typedef struct {
  int64_t r2;
  int32_t dx, dy;
} disp_t;

static int disp_cmp(const void* a, const void* b) {
  const disp_t* p = (const disp_t*)a;
  const disp_t* q = (const disp_t*)b;
  if (p->r2 != q->r2) return p->r2 < q->r2 ? -1 : 1;
  if (p->dy != q->dy) return p->dy < q->dy ? -1 : 1;
  if (p->dx != q->dx) return p->dx < q->dx ? -1 : 1;
  return 0;
}

int sco_ref_table(int32_t Lx, int32_t Ly, int32_t* dx, int32_t* dy, int64_t* r2, double* c,
                  uint64_t* A, uint64_t* W) {
  int64_t K = sco_ref_table_size(Lx, Ly);
  if (K < 0) return SCO_REF_EINVAL;
  if (K == 0) return SCO_REF_OK;
  disp_t* d = (disp_t*)malloc((size_t)K * sizeof(disp_t));
  if (!d) return SCO_REF_ENOMEM;
  int64_t n = 0;
  for (int32_t y = 0; y < Ly; ++y) {
    for (int32_t x = -(Lx - 1); x <= Lx - 1; ++x) {
      if (y == 0 && x <= 0) continue;
      d[n].dx = x;
      d[n].dy = y;
      d[n].r2 = (int64_t)x * x + (int64_t)y * y;
      ++n;
    }
  }
  qsort(d, (size_t)K, sizeof(disp_t), disp_cmp);
  uint64_t acc = 0;
  for (int64_t m = 0; m < K; ++m) {
    uint64_t a = ref_hazard_A(d[m].r2);
    acc += a;
    if (dx) dx[m] = d[m].dx;
    if (dy) dy[m] = d[m].dy;
    if (r2) r2[m] = d[m].r2;
    if (c) c[m] = ref_coupling_c(d[m].r2);
    if (A) A[m] = a;
    if (W) W[m] = acc;
  }
  free(d);
  return SCO_REF_OK;
}
