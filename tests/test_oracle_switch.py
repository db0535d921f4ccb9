"""Pins of the oracle's potential switching (Sec. 2.1 step (A)).

The bound-thinned O(N) switch must make every pair survive independently with probability
1 - P_ij (Eq. (2)).  Checked per pair against that probability, against the direct O(N^2)
definition, against the closed form for independent uniform spins, and against Table 1.
"""
import os

import numpy as np
import pytest

import oracle as O
from switch_theory import expected_edges

HERE = os.path.dirname(os.path.abspath(__file__))


def _exact_survival(params, xyz):
    """1 - P_ij for every pair i < j from the textbook dipolar formula (numpy, FP64)."""
    Lx, Ly = params.Lx, params.Ly
    N = Lx * Ly
    S = xyz.reshape(3, N).T
    pos = np.stack([np.arange(N) % Lx, np.arange(N) // Lx], 1).astype(float)
    beta = 1.0 / params.T
    out = {}
    for i in range(N):
        for j in range(i + 1, N):
            d = np.array([*(pos[j] - pos[i]), 0.0])
            r = np.linalg.norm(d)
            V = params.D * (S[i] @ S[j] / r ** 3 - 3 * (S[i] @ d) * (S[j] @ d) / r ** 5)
            vm = O.vmax(params.D, int(round(r * r)))
            out[(i, j)] = 1.0 - np.exp(beta * (V - vm))
    return out


def test_thinned_switch_is_exact_per_pair():
    p = O.make_params(4, T=0.5, seed=7)
    ch = O.Chain(p)
    exact = _exact_survival(p, ch.spins())
    n_epochs = 6000
    counts = {k: 0 for k in exact}
    for e in range(n_epochs):
        ch.switch_epoch(e)
        i, j, m, f = ch.edges()
        for a, b in zip(i.tolist(), j.tolist()):
            counts[(a, b)] += 1
    z = []
    for k, q in exact.items():
        sd = np.sqrt(max(q * (1 - q), 1e-12) * n_epochs)
        z.append((counts[k] - q * n_epochs) / sd)
    z = np.array(z)
    assert np.all(np.abs(z) < 5.0)
    assert abs(z.mean()) < 5.0 / np.sqrt(len(z))  # no common bias
    assert 0.5 < (z ** 2).mean() < 1.6


def test_direct_switch_agrees_with_probabilities():
    p = O.make_params(3, 3, T=0.4, seed=2)
    ch = O.Chain(p)
    exact = _exact_survival(p, ch.spins())
    n = 4000
    acc = np.zeros((9, 9))
    for e in range(n):
        acc += ch.direct_switch(e)
    for (i, j), q in exact.items():
        assert abs(acc[i, j] - q * n) < 5 * np.sqrt(max(q * (1 - q), 1e-12) * n)


@pytest.mark.parametrize("T", [0.3, 0.6, 1.2])
def test_mean_degree_matches_closed_form(T):
    L = 192
    p = O.make_params(L, T=T, seed=3)
    ch = O.Chain(p)
    got = []
    for e in range(2):
        ch.switch_epoch(e)
        got.append(ch.observables()["n_edges"])
    exp = expected_edges(L, L, 1.0 / T)
    assert abs(np.mean(got) - exp) < 0.01 * exp


def _table1():
    rows = []
    for line in open(os.path.join(HERE, "golden", "table1_degrees.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append([float(x) for x in line.split()])
    return rows


def test_table1_paramagnetic_row():
    # Table 1, T = 1.25J (D/J = 0.1, beta D = 0.08): well above T_c = 0.88J the spins are
    # close to independent, so the closed form for independent uniform spins applies.
    T_J, k_paper, delta_paper = _table1()[0]
    betaD = 0.1 / T_J
    L = 1024
    p = O.make_params(L, T=1.0 / betaD, seed=5)
    ch = O.Chain(p)
    ch.switch_epoch(0)
    o = ch.observables()
    k = 2 * o["n_edges"] / (L * L)
    k_theory = 2 * expected_edges(L, L, betaD) / (L * L)
    assert abs(k - k_theory) < 0.01                # oracle vs closed form (sampling noise ~0.002)
    assert abs(k_theory - k_paper) < 0.06          # reading vs the printed value
    assert abs(o["max_degree_dipolar"] - delta_paper) <= 2.5
