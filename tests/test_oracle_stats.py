"""Pins of the oracle's graph diagnostics (Sec. 3.2, Figs. 5 and 6; Sec. 3.3, Eq. (9)) and of its
temperature change (the cooling protocol of Sec. 3.1).

P_survive(r): the pair counts per distance shell against a brute-force count over all site
pairs; the survival fraction per shell against the closed form for independent uniform spins.
P_IPC: the one-cell and one-site-per-cell limits and a numpy recount of the oracle's edge list.
Delta R of Eq. (9): zero for one cell, and a numpy recount of the oracle's colours."""
import math

import numpy as np
import pytest

import oracle as O
from switch_theory import survival


def _chain(L, T, seed, J=0.0, D=1.0, Ly=None):
    ch = O.Chain(O.make_params(L, Ly, T=T, J=J, D=D, seed=seed))
    ch.switch()
    ch.colour()
    return ch


def _shell(r2, nb):
    return min(math.isqrt(r2) - 1, nb - 1)


@pytest.mark.parametrize("Lx,Ly,nb", [(9, 7, 6), (12, 12, 40), (5, 1, 3), (1, 1, 2)])
def test_pair_counts_per_shell_brute_force(Lx, Ly, nb):
    ch = _chain(Lx, 0.5, 1, Ly=Ly)
    st = ch.graph_stats(1, 1, nb)
    N = Lx * Ly
    want = np.zeros(nb, np.int64)
    for i in range(N):
        for j in range(i + 1, N):
            dx, dy = j % Lx - i % Lx, j // Lx - i // Lx
            want[_shell(dx * dx + dy * dy, nb)] += 1
    assert np.array_equal(st["pairs"], want)
    assert st["pairs"].sum() == N * (N - 1) // 2
    assert st["survived"].sum() == st["n_pairs"] == ch.observables()["n_edges"]


def test_survival_per_shell_matches_closed_form():
    # random-start spins are iid uniform: the expected survival fraction of a shell is the
    # pair-count-weighted mean of the closed form s(beta D / r^3) over its displacements
    L, T, nb = 64, 0.5, 6
    betaD = 1.0 / T
    ch = O.Chain(O.make_params(L, T=T, seed=9))
    surv = np.zeros(nb)
    n_graphs = 6
    for e in range(n_graphs):
        ch.switch_epoch(e)
        ch.colour()
        st = ch.graph_stats(1, 1, nb)
        surv += st["survived"]
    pairs = st["pairs"]
    expect = np.zeros(nb)
    for dy in range(L):
        for dx in range(-(L - 1), L):
            if dy == 0 and dx <= 0:
                continue
            r2 = dx * dx + dy * dy
            expect[_shell(r2, nb)] += (L - abs(dx)) * (L - dy) * survival(betaD / r2 ** 1.5)
    for b in range(nb):
        m = expect[b] * n_graphs
        # pairs of one graph share spins, so allow a generous 6 sigma of the binomial spread
        assert abs(surv[b] - m) < 6 * math.sqrt(m * n_graphs) + 1e-9, (b, surv[b], m)
    ps = st["p_survive"]
    assert np.all((ps >= 0) & (ps <= 1))
    assert ps[0] > ps[1] > ps[2]  # survival falls with distance (Fig. 5)


def test_cross_cell_fraction_limits_and_recount():
    L = 24
    ch = _chain(L, 0.4, 3)
    assert ch.graph_stats(1, 1, 8)["n_cross"] == 0
    st = ch.graph_stats(L, L, 8)  # every site its own cell: every pair crosses
    assert st["n_cross"] == st["n_pairs"] and st["p_ipc"] == 1.0
    i, j, _, f = ch.edges()
    dip = (f & 1) == 1
    i, j = i[dip], j[dip]
    for cx, cy in [(2, 1), (3, 4), (5, 7)]:
        cell = lambda s: (s % L) * cx // L + cx * ((s // L) * cy // L)
        want = int(np.sum(cell(i) != cell(j)))
        st = ch.graph_stats(cx, cy, 8)
        assert st["n_cross"] == want and st["n_cells"] == cx * cy
        assert st["p_ipc"] == want / len(i)


def test_colour_imbalance_one_cell_and_recount():
    L = 30
    ch = _chain(L, 0.5, 4)
    st = ch.graph_stats(1, 1, 4)
    assert np.all(np.nan_to_num(st["delta_r"]) == 0.0) and st["delta_r_mean"] == 0.0
    col = ch.colours()
    x, y = np.arange(L * L) % L, np.arange(L * L) // L
    for cx, cy in [(2, 2), (3, 5), (30, 1)]:
        cell = x * cx // L + cx * (y * cy // L)
        st = ch.graph_stats(cx, cy, 4)
        drs = []
        for c in range(st["palette"]):
            k = np.bincount(cell[col == c], minlength=cx * cy)
            if k.sum() == 0:
                assert np.isnan(st["delta_r"][c])
                continue
            kave = k.sum() / (cx * cy)
            drs.append((k.max() - kave) / kave)
            assert st["delta_r"][c] == pytest.approx(drs[-1], rel=1e-15)
        assert st["delta_r_mean"] == pytest.approx(np.mean(drs), rel=1e-14)
        assert st["delta_r_max"] == pytest.approx(np.max(drs), rel=1e-15)
        # class-size weighted: sum_c |c| Delta R_c / N = cells sum_c K_max,c / N - 1
        kmax = [np.bincount(cell[col == c], minlength=cx * cy).max() for c in range(st["palette"])]
        assert st["delta_r_weighted"] == pytest.approx(cx * cy * sum(kmax) / (L * L) - 1,
                                                       rel=1e-14, abs=1e-15)
    assert ch.graph_stats(1, 1, 4)["delta_r_weighted"] == 0.0


def test_set_temperature_rebuilds_the_graph_at_the_new_beta():
    # After a temperature change the next MC step switches again (same epoch number) with the
    # new beta: the trajectory equals one that starts from the same spins at the new T with the
    # step counter carried over, and a hotter lattice keeps fewer pairs (Eq. (2)).
    L = 20
    a = O.Chain(O.make_params(L, T=0.4, J=1.0, D=0.1, seed=5, n_sw=3))
    a.sweep(4)
    k_cold = a.observables()["n_edges"]
    a.set_temperature(5.0)
    a.sweep(1)
    k_hot = a.observables()["n_edges"]
    assert k_hot < k_cold
    # the switch after the change equals the switch of a lattice created at the new T with the
    # same spins and epoch (the switch is a function of spins, epoch, beta and seed only)
    b = O.Chain(O.make_params(L, T=5.0, J=1.0, D=0.1, seed=5, n_sw=3))
    for T2 in (0.7, 5.0):
        a.set_temperature(T2)
        b.set_temperature(T2)
        b.set_spins(a.spins())
        a.switch_epoch(7)
        b.switch_epoch(7)
        ra, ca = a.graph()
        rb, cb = b.graph()
        assert np.array_equal(ra, rb) and np.array_equal(ca, cb)
    fresh = O.Chain(O.make_params(L, T=0.7, J=1.0, D=0.1, seed=5, n_sw=3))
    fresh.set_spins(a.spins())
    fresh.switch_epoch(7)
    a.set_temperature(0.7)
    a.switch_epoch(7)
    assert np.array_equal(fresh.graph()[1], a.graph()[1])
    with pytest.raises(RuntimeError):
        a.set_temperature(-1.0)
