/* ref_internal.h -- helpers shared by the oracle's own C files (test infrastructure only). */
#ifndef SCO_REF_INTERNAL_H
#define SCO_REF_INTERNAL_H

#include <stdint.h>

#include "sco_ref.h"

typedef long double hp_t; /* extended precision for near-tie decisions */

/* c(r^2) = fl(1 / (fl(r2*r2) * fl(sqrt(r2)))), the FP64 constant that stands for r^-5. */
double ref_coupling_c(int64_t r2);
/* A(r^2) = trunc(fl(fl(2^60 / fl(r2 * sqrt(r2))) * (1 + 2^-50))) + 1 > 2^60 / r^3. */
uint64_t ref_hazard_A(int64_t r2);
/* V of Eq. (6) for one pair, FP64, with the displacement d = (dx, dy, 0) from i to j. */
double ref_V(double D, double c, int64_t r2, const double Si[3], const double Sj[3], int32_t dx,
             int32_t dy);
hp_t ref_V_hp(double D, double c, int64_t r2, const double Si[3], const double Sj[3], int32_t dx,
              int32_t dy);
/* log(1 - e^x) for x < 0 (Maechler 2012); *sens receives an upper bound of e^x / (1 - e^x). */
double ref_log1mexp(double x, double* sens);
hp_t ref_log1mexp_hp(hp_t x);

#endif
