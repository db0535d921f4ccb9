"""Closed forms for the switching statistics of independent uniform spins (test helper).

For unit spins drawn independently and uniformly on the sphere, the dipolar pair energy in
units of D/r^3 is v = S_i.w with w = S_j - 3 (S_j.r^) r^, |w|^2 = 1 + 3 t^2, t = S_j.r^
uniform on [-1, 1] (Archimedes).  Averaging exp(lambda S_i.w) over S_i gives
sinh(lambda |w|) / (lambda |w|), so with lambda = beta D / r^3 and V_max = 2D / r^3 the
survival probability 1 - P_ij of Eq. (2) averages to
    s(lambda) = 1 - exp(-2 lambda) * int_0^1 sinh(lambda q) / (lambda q) dt,  q = sqrt(1 + 3 t^2).
"""
import numpy as np
from scipy.integrate import quad


def survival(lam):
    if lam < 1e-6:
        return 2 * lam - (7.0 / 3.0) * lam * lam
    f = quad(lambda t: np.sinh(lam * np.sqrt(1 + 3 * t * t)) / (lam * np.sqrt(1 + 3 * t * t)),
             0.0, 1.0, epsabs=1e-14, epsrel=1e-12)[0]
    return 1.0 - np.exp(-2 * lam) * f


def expected_edges(Lx, Ly, betaD):
    """Expected number of surviving pairs on the open Lx x Ly lattice for iid uniform spins."""
    cache = {}
    total = 0.0
    for dy in range(0, Ly):
        for dx in range(-(Lx - 1), Lx):
            if dy == 0 and dx <= 0:
                continue
            r2 = dx * dx + dy * dy
            if r2 not in cache:
                cache[r2] = survival(betaD / r2 ** 1.5)
            total += cache[r2] * (Lx - abs(dx)) * (Ly - dy)
    return total
