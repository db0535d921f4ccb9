/*
 * ref_rng.c -- oracle random numbers.  TEST INFRASTRUCTURE ONLY (see sco_ref.h).
 *
 * The paper names no generator; the random numbers of the method are drawn
 * from a counter-based generator keyed by (seed, replica) with counter
 * (site, step, draw, tag), so that every draw is addressable and the CPU and
 * GPU trajectories coincide.
 */
#include <math.h>

#include "sco_ref.h"

/* Philox4x64 with 10 rounds, as defined by Salmon, Moraes, Dror and Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3" (SC'11): each round multiplies
 * counter words 0 and 2 by the two round multipliers, mixes the high halves
 * with the other counter words and the key, and the key is bumped by the two
 * Weyl increments between rounds. */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ull;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ull;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ull;
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73Bull;

void sco_ref_philox(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    unsigned __int128 p0 = (unsigned __int128)PHILOX_M0 * c0;
    unsigned __int128 p1 = (unsigned __int128)PHILOX_M1 * c2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* Marsaglia (1972), "Choosing a point from the surface of a sphere":
 * a1, a2 uniform on (-1, 1); reject unless 0 < s = a1^2 + a2^2 < 1; then
 * S = (2 a1 sqrt(1-s), 2 a2 sqrt(1-s), 1 - 2 s).  Uniforms are u = (w >> 11) 2^-53,
 * so a = 2u - 1 is exact.  Only correctly rounded + - * sqrt are used, each
 * rounded on its own (the oracle is compiled without contraction). */
int sco_ref_marsaglia(uint64_t w0, uint64_t w1, double S[3]) {
  double u0 = (double)(w0 >> 11) * 0x1p-53;
  double u1 = (double)(w1 >> 11) * 0x1p-53;
  double a1 = 2.0 * u0 - 1.0;
  double a2 = 2.0 * u1 - 1.0;
  double s = a1 * a1 + a2 * a2;
  if (s >= 1.0 || s == 0.0) return 0;
  double h = sqrt(1.0 - s);
  S[0] = (2.0 * a1) * h;
  S[1] = (2.0 * a2) * h;
  S[2] = 1.0 - 2.0 * s;
  return 1;
}
