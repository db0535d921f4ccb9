"""Pins of the oracle's model pieces: coupling table, dipolar potential, V_max,
switching probability and pseudointeraction (Sec. 2.1 Eqs. (1)-(3), Sec. 3.1 Eq. (6))."""
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle as O

getcontext().prec = 60


@pytest.mark.parametrize("Lx,Ly", [(1, 1), (2, 1), (1, 3), (4, 4), (5, 3), (3, 7), (16, 16)])
def test_table_lists_every_pair_once(Lx, Ly):
    t = O.table(Lx, Ly)
    K = len(t["dx"])
    assert K == (Lx - 1) + (Ly - 1) * (2 * Lx - 1)
    disp = set(zip(t["dx"].tolist(), t["dy"].tolist()))
    assert len(disp) == K
    # brute force: every unordered pair of sites maps to exactly one listed displacement
    N = Lx * Ly
    seen = {}
    for i in range(N):
        for j in range(i + 1, N):
            dx, dy = j % Lx - i % Lx, j // Lx - i // Lx
            d = (dx, dy) if (dy > 0 or (dy == 0 and dx > 0)) else (-dx, -dy)
            assert d in disp
            seen[d] = seen.get(d, 0) + 1
    # every listed displacement occurs in (Lx - |dx|)(Ly - |dy|) pairs
    for dx, dy in disp:
        assert seen.get((dx, dy), 0) == (Lx - abs(dx)) * (Ly - abs(dy))


def test_table_order_and_square_size():
    L = 9
    t = O.table(L)
    assert len(t["dx"]) == ((2 * L - 1) ** 2 - 1) // 2
    key = list(zip(t["r2"].tolist(), t["dy"].tolist(), t["dx"].tolist()))
    assert key == sorted(key)
    assert np.all(t["r2"] == t["dx"].astype(np.int64) ** 2 + t["dy"].astype(np.int64) ** 2)


def test_coupling_constant_is_r_minus_5_within_two_ulp():
    t = O.table(40)
    for r2, c in zip(t["r2"][::7].tolist(), t["c"][::7].tolist()):
        exact = 1 / (Decimal(r2) ** 2 * Decimal(r2).sqrt())
        rel = abs((Decimal(c) - exact) / exact)
        assert rel <= Decimal(3) * Decimal(2) ** -53


def test_hazard_bounds_max_dipolar_energy_exactly():
    # V_max = D A 2^-59 must be >= 2D/r^3, i.e. A >= 2^60 / r^3, i.e. A^2 r2^3 >= 2^120
    # (integers, exact); and the slack is tiny: A <= 2^60/r^3 (1 + 2^-48) + 2.
    t = O.table(64)
    for r2, A in zip(t["r2"].tolist(), t["A"].tolist()):
        assert A * A * r2 ** 3 >= 2 ** 120
        bound = Decimal(2) ** 60 / (Decimal(r2) * Decimal(r2).sqrt())
        assert Decimal(A) <= bound * (1 + Decimal(2) ** -48) + 2
    W = t["W"].tolist()
    acc = 0
    for a, w in zip(t["A"].tolist(), W):
        acc += a
        assert w == acc
    assert acc < 2 ** 63


def test_total_hazard_matches_lattice_sum():
    # twice the half-plane sum of A 2^-60 ~ r^-3 is the sum over the square |dx|,|dy| <= L-1 of r^-3;
    # the infinite-lattice sum is 4 zeta(3/2) beta(3/2) (beta: Dirichlet beta, via Hurwitz
    # zeta), and the part outside a square of half-side a is 4 sqrt(2) / a to first order.
    from scipy.special import zeta
    lattice = 4 * zeta(1.5) * 4 ** -1.5 * (zeta(1.5, 0.25) - zeta(1.5, 0.75))
    L = 200
    t = O.table(L)
    total = 2 * int(t["W"][-1]) * 2.0 ** -60  # half plane counts each pair once
    expected = lattice - 4 * np.sqrt(2) / (L - 0.5)
    assert abs(total - expected) < 2e-4


def _rand_unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_dipolar_potential_closed_forms():
    D = 1.7
    x, y, z = np.eye(3)
    for dx, dy in [(1, 0), (0, 1), (3, 4), (-5, 2)]:
        r = np.hypot(dx, dy)
        rh = np.array([dx, dy, 0.0]) / r
        # spins along the bond, parallel: V = D (1 - 3) / r^3
        assert O.pair_V(D, rh, rh, dx, dy) == pytest.approx(-2 * D / r ** 3, rel=1e-14)
        # antiparallel along the bond reaches the maximum 2D / r^3
        assert O.pair_V(D, rh, -rh, dx, dy) == pytest.approx(2 * D / r ** 3, rel=1e-14)
        # both out of plane: V = D / r^3; orthogonal in-plane pair along/perp: 0
        assert O.pair_V(D, z, z, dx, dy) == pytest.approx(D / r ** 3, rel=1e-14)
        perp = np.array([-rh[1], rh[0], 0.0])
        assert abs(O.pair_V(D, rh, perp, dx, dy)) < 1e-15 * D / r ** 3 * 10


def test_vmax_dominates_every_pair():
    rng = np.random.default_rng(11)
    Si, Sj = _rand_unit(rng, 20000), _rand_unit(rng, 20000)
    for dx, dy in [(1, 0), (1, 1), (2, 1), (7, 3), (0, 12)]:
        r2 = dx * dx + dy * dy
        vm = O.vmax(1.0, r2)
        V = np.array([O.pair_V(1.0, a, b, dx, dy) for a, b in zip(Si[:4000], Sj[:4000])])
        assert V.max() < vm
        assert vm >= 2 / r2 ** 1.5 and vm <= 2 / r2 ** 1.5 * (1 + 2 ** -45)
        assert V.max() > 0.8 * 2 / r2 ** 1.5  # the sup 2D/r^3 is approached


def test_sps_identity_and_probability_range():
    # Eqs. (2)-(3): exp(-beta Vbar) = exp(-beta V) (1 - P), hence
    # exp(-beta Vbar) + exp(-beta Vmax) = exp(-beta V), with P in (0, 1].
    rng = np.random.default_rng(5)
    for beta in [0.08, 0.5, 1.0, 5.0]:
        for r2 in [1, 2, 5, 50]:
            vm = O.vmax(1.0, r2)
            for V in rng.uniform(-vm, vm * (1 - 1e-9), size=200):
                P = O.switch_prob(beta, V, vm)
                assert 0.0 < P <= 1.0
                vb = O.pseudo(beta, V, vm)
                lhs = np.exp(-beta * vb) + np.exp(-beta * vm)
                assert lhs == pytest.approx(np.exp(-beta * V), rel=1e-13)
