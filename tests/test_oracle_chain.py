"""Pins of the oracle's whole SCO chain (Sec. 2.1 steps (A)-(C), Fig. 1).

The SCO method samples the exact Boltzmann distribution of H (Eq. (6)): checked on a
two-spin system against the exact energy density, and on 4x4 / 8x8 lattices against a
plain full-interaction Metropolis run.  Special cases: beta -> 0, D = 0.  Observables are
checked against closed forms."""
import numpy as np
import pytest

import oracle as O


def _binned(x, nbins=40):
    b = len(x) // nbins
    means = x[: b * nbins].reshape(nbins, b).mean(1)
    return means.mean(), means.std(ddof=1) / np.sqrt(nbins)


def test_two_spin_energy_density_is_boltzmann():
    # Two spins at distance 1 along x, J = 0, D = 1, beta = 2.  Exact density of V is
    # g(V) exp(-beta V); bin probabilities from independent numpy samples of uniform spin
    # pairs weighted by exp(-beta V) (textbook dipolar formula).
    beta = 2.0
    rng = np.random.default_rng(123)
    n_ref = 4_000_000
    a = rng.normal(size=(n_ref, 3)); a /= np.linalg.norm(a, axis=1, keepdims=True)
    b = rng.normal(size=(n_ref, 3)); b /= np.linalg.norm(b, axis=1, keepdims=True)
    v = (a * b).sum(1) - 3 * a[:, 0] * b[:, 0]
    w = np.exp(-beta * v)
    edges = np.linspace(-2, 2, 17)
    ref, _ = np.histogram(v, bins=edges, weights=w)
    ref /= ref.sum()
    O.set_threads(1)
    ch = O.Chain(O.make_params(2, 1, T=1 / beta, seed=4))
    e, _ = ch.run_series(300_000)
    V = 2 * e[1000::6]  # E/N with N = 2; thinned against autocorrelation
    hist, _ = np.histogram(V, bins=edges)
    n = hist.sum()
    expct = ref * n
    keep = expct > 20
    chi2 = ((hist[keep] - expct[keep]) ** 2 / expct[keep]).sum()
    dof = keep.sum() - 1
    # p > 1e-3 for chi2 with ~15 dof means chi2 < ~37.7
    assert chi2 < 37.7, (chi2, dof)
    # mean energy within 4 binned standard errors of the exact mean
    m, s = _binned(2 * e[1000:])
    assert abs(m - (v * w).sum() / w.sum()) < 4 * s + 2e-3


@pytest.mark.parametrize("L,T,J,D,n", [(4, 0.8, 0.0, 1.0, 120_000), (8, 0.8, 0.0, 1.0, 50_000),
                                       (4, 1.0, 1.0, 0.1, 100_000)])
def test_equilibrium_matches_plain_metropolis(L, T, J, D, n):
    O.set_threads(1)
    p = O.make_params(L, T=T, J=J, D=D, seed=11)
    ch = O.Chain(p)
    e1, m1 = ch.run_series(n)
    q = O.make_params(L, T=T, J=J, D=D, seed=12)
    e2, m2, _ = O.plain_metropolis(q, ch.spins(), n)
    burn = n // 20
    for x1, x2 in ((e1, e2), (m1, m2)):
        a, sa = _binned(x1[burn:])
        b, sb = _binned(x2[burn:])
        assert abs(a - b) < 3 * np.hypot(sa, sb), (a, b, sa, sb)


def test_infinite_temperature_accepts_everything():
    ch = O.Chain(O.make_params(12, T=1e12, seed=3))
    ch.sweep(1)
    o = ch.observables()
    assert o["n_edges"] == 0 and o["max_degree"] == 0 and o["n_colours"] == 1
    assert np.all(ch.accepts() == 1)


def test_exchange_only_graph_is_the_lattice():
    L = 6
    ch = O.Chain(O.make_params(L, T=0.7, J=1.0, D=0.0, seed=3))
    ch.sweep(2)
    rp, col = ch.graph()
    assert np.all(col & O.EXCH_ONLY)  # no dipolar pair survives when D = 0
    deg = np.diff(rp)
    x, y = np.arange(L * L) % L, np.arange(L * L) // L
    assert np.array_equal(deg, 4 - (x == 0) - (x == L - 1) - (y == 0) - (y == L - 1))
    colour = ch.colours()
    for i in range(L * L):
        for j in col[rp[i]:rp[i + 1]] & 0x7FFFFFFF:
            assert colour[i] != colour[j]
            assert abs(int(j) - i) in (1, L)


def test_thread_count_does_not_change_the_trajectory():
    out = []
    for nt in (1, 3):
        O.set_threads(nt)
        ch = O.Chain(O.make_params(24, T=0.5, seed=8))
        ch.sweep(3)
        out.append(ch.spins())
    O.set_threads(0)
    assert np.array_equal(out[0], out[1])


def test_observables_closed_forms():
    L = 6
    ch = O.Chain(O.make_params(L, T=0.5, seed=1))
    x, y = np.arange(L * L) % L, np.arange(L * L) // L
    ux, uy = x - (L - 1) / 2, y - (L - 1) / 2
    r = np.hypot(ux, uy)
    # vortex: S = z x u^  ->  [S x u^]_z = -1 at every site (Eq. (7))
    ch.set_spins(np.concatenate([-uy / r, ux / r, np.zeros(L * L)]))
    o = ch.observables(full=True)
    assert o["m_phi"] == pytest.approx(-1.0, abs=1e-14)
    assert o["m_abs"] < 1e-14
    # all spins along z: every pair contributes D / r^3 (Eq. (6))
    ch.set_spins(np.concatenate([np.zeros(2 * L * L), np.ones(L * L)]))
    o = ch.observables(full=True)
    pairs = 0.0
    for i in range(L * L):
        for j in range(i + 1, L * L):
            pairs += np.hypot(x[j] - x[i], y[j] - y[i]) ** -3
    assert o["e_full"] == pytest.approx(pairs, rel=1e-13)
    assert o["m_abs"] == pytest.approx(1.0) and o["mz"] == pytest.approx(1.0)


def test_two_spin_switched_energy():
    beta = 1.5
    ch = O.Chain(O.make_params(2, 1, T=1 / beta, seed=2))
    for e in range(50):
        ch.switch_epoch(e)
        o = ch.observables(full=True)
        if o["n_edges"]:
            break
    assert o["n_edges"] == 1
    s = ch.spins().reshape(3, 2)
    V = s[:, 0] @ s[:, 1] - 3 * s[0, 0] * s[0, 1]
    vm = O.vmax(1.0, 1)
    vbar = V - np.log1p(-np.exp(beta * (V - vm))) / beta
    assert o["e_switched"] == pytest.approx(vbar, rel=1e-13)
    assert o["e_full"] == pytest.approx(V, rel=1e-13, abs=1e-15)


def test_extended_precision_path_gives_the_same_trajectory():
    # Every decision is an exact real comparison; FP64 with its error bound and the
    # extended-precision re-evaluation must agree.  Force the latter everywhere.
    runs = []
    for scale in (1.0, 1e280):
        O.set_guard_scale(scale)
        ch = O.Chain(O.make_params(10, T=0.4, J=0.3, seed=21))
        ch.sweep(6)
        o = ch.observables()
        runs.append((ch.spins(), o["guard_hits"]))
    O.set_guard_scale(1.0)
    assert np.array_equal(runs[0][0], runs[1][0])
    assert runs[1][1] > 1000 * max(runs[0][1], 1)


def _bond_count(Lx, Ly):
    # open Lx x Ly lattice: Ly rows of Lx - 1 horizontal bonds, Lx columns of Ly - 1 vertical
    return Lx * (Ly - 1) + Ly * (Lx - 1)


@pytest.mark.parametrize("Lx,Ly,J", [(5, 3, 1.0), (1, 6, 0.7), (4, 4, -2.5), (7, 1, 1.0)])
def test_exchange_energy_closed_forms(Lx, Ly, J):
    # The exchange term of Eq. (6), -J sum_<ij> S_i.S_j over nearest-neighbour bonds.
    # All spins parallel: every bond gives -J.  Neel checkerboard along z: every bond joins
    # opposite spins (+J).  In-plane spins alternating between +x and +y by column: the
    # horizontal bonds are orthogonal (0) and the vertical bonds parallel (-J each).
    N = Lx * Ly
    x, y = np.arange(N) % Lx, np.arange(N) // Lx
    nb = _bond_count(Lx, Ly)
    ch = O.Chain(O.make_params(Lx, Ly, T=0.5, J=J, seed=1))
    ch.set_spins(np.concatenate([np.zeros(2 * N), np.ones(N)]))
    assert ch.observables()["e_exchange"] == pytest.approx(-J * nb, rel=1e-15)
    sz = np.where((x + y) % 2 == 0, 1.0, -1.0)
    ch.set_spins(np.concatenate([np.zeros(2 * N), sz]))
    assert ch.observables()["e_exchange"] == pytest.approx(J * nb, rel=1e-15)
    even = (x % 2 == 0).astype(float)
    ch.set_spins(np.concatenate([even, 1.0 - even, np.zeros(N)]))
    assert ch.observables()["e_exchange"] == pytest.approx(-J * Lx * (Ly - 1), rel=1e-15,
                                                           abs=1e-15)


def test_exchange_energy_brute_force_neighbour_search():
    # Random spins on a 4 x 3 lattice: the exchange energy against a sum over every pair of
    # sites whose displacement has |dx| + |dy| = 1 (an independent neighbour search).
    Lx, Ly, J = 4, 3, 1.3
    N = Lx * Ly
    rng = np.random.default_rng(5)
    s = rng.normal(size=(N, 3))
    s /= np.linalg.norm(s, axis=1, keepdims=True)
    x, y = np.arange(N) % Lx, np.arange(N) // Lx
    e = 0.0
    for i in range(N):
        for j in range(i + 1, N):
            if abs(int(x[j]) - int(x[i])) + abs(int(y[j]) - int(y[i])) == 1:
                e -= J * float(s[i] @ s[j])
    ch = O.Chain(O.make_params(Lx, Ly, T=0.5, J=J, seed=2))
    ch.set_spins(s.T.reshape(-1))
    assert ch.observables()["e_exchange"] == pytest.approx(e, rel=1e-14)


def test_two_spin_exchange_and_switched_energy():
    # A 2 x 1 lattice with J != 0: e_exchange = -J S_1.S_2 exactly, and the switched energy
    # H' of Eq. (4) adds the pseudointeraction Vbar of Eq. (3) when the dipolar pair survives.
    # With D = 0 the exchange bond is the only term (no pair can survive).
    beta, J = 1.5, 0.8
    for D in (1.0, 0.0):
        ch = O.Chain(O.make_params(2, 1, T=1 / beta, J=J, D=D, seed=2))
        seen = set()
        for e in range(80):
            ch.switch_epoch(e)
            o = ch.observables(full=True)
            s = ch.spins().reshape(3, 2)
            dot = float(s[:, 0] @ s[:, 1])
            assert o["e_exchange"] == pytest.approx(-J * dot, rel=1e-15)
            V = D * (dot - 3 * s[0, 0] * s[0, 1])
            vbar = 0.0
            if o["n_edges"]:
                vm = O.vmax(D, 1)
                vbar = V - np.log1p(-np.exp(beta * (V - vm))) / beta
            assert o["e_switched"] == pytest.approx(vbar - J * dot, rel=1e-13)
            assert o["e_full"] == pytest.approx(V - J * dot, rel=1e-13, abs=1e-15)
            seen.add(o["n_edges"])
            if D == 0.0:
                assert o["n_edges"] == 0
            ch.sweep(1)
        if D == 1.0:
            assert seen == {0, 1}  # both switch outcomes were exercised
