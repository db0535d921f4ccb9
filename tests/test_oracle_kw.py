"""Pins of the oracle's Kuhn-Wattenhofer colouring (Sec. 2.3).

Checked: validity (no edge inside a colour class), palette [0, Delta] (Sec. 2.3.1), running
time t_R <= (Delta + 1) M (Eq. (5)) and = (Delta + 1) M for plain BCR, cliques, empty graphs,
and an independent sequential evaluation (see _dependency_order)."""
import numpy as np
import pytest

import oracle as O
import graphs as G


def _check_valid(rp, col, colour, delta):
    n = len(rp) - 1
    assert colour.min(initial=0) >= 0 and colour.max(initial=0) <= delta
    for i in range(n):
        for j in col[rp[i]:rp[i + 1]]:
            assert colour[i] != colour[int(j)]


def _levels(n, delta):
    g = delta + 1
    groups = -(-n // g) if n else 0
    M = 0
    while (1 << M) < groups:
        M += 1
    return M


def _dependency_order(rp, col):
    """Sequential restatement: at every level the right-half vertices are recoloured one at a
    time in decreasing colour, each taking the smallest colour no same-group neighbour holds.
    A vertex recoloured by a synchronous round of step (2)' has seen exactly the final colours
    of its larger-coloured neighbours and the unchanged colours (>= Delta+1) of the rest, so
    both orders give the same colouring."""
    n = len(rp) - 1
    delta = int(np.max(np.diff(rp))) if n else 0
    g = delta + 1
    lc = [i % g for i in range(n)]
    for p in range(1, _levels(n, delta) + 1):
        right = [i for i in range(n) if ((i // g) >> (p - 1)) & 1]
        for i in right:
            lc[i] += g
        for v in sorted(right, key=lambda v: -lc[v]):
            used = {lc[int(u)] for u in col[rp[v]:rp[v + 1]] if (int(u) // g) >> p == (v // g) >> p}
            lc[v] = min(c for c in range(g) if c not in used)
    return np.array(lc, np.int32)


CASES = [
    ("er_sparse", lambda: G.erdos_renyi(300, 0.02, 1)),
    ("er_dense", lambda: G.erdos_renyi(120, 0.2, 2)),
    ("geometric", lambda: G.geometric(400, 0.09, 3)),
    ("geometric_shuffled", lambda: G.shuffled(400, *G.geometric(400, 0.09, 4), 5)),
    ("lattice", lambda: G.lattice(13, 9)),
    ("path", lambda: G.path(50)),
    ("star", lambda: G.star(33)),
    ("clique", lambda: G.clique(9)),
    ("empty", lambda: G.empty(37)),
    ("single", lambda: G.empty(1)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_kw_valid_bounded_and_schedule_free(name, make):
    rp, col = make()
    n = len(rp) - 1
    colour, rounds, delta = O.kw_colour_graph(rp, col, variant=0)
    assert delta == (int(np.max(np.diff(rp))) if n else 0)
    _check_valid(rp, col, colour, delta)
    M = _levels(n, delta)
    assert rounds <= (delta + 1) * M
    plain, rounds_plain, _ = O.kw_colour_graph(rp, col, variant=1)
    assert np.array_equal(plain, colour)
    assert rounds_plain == (delta + 1) * M
    assert np.array_equal(_dependency_order(rp, col), colour)


def test_clique_uses_every_colour():
    for n in (2, 5, 12):
        rp, col = G.clique(n)
        colour, _, delta = O.kw_colour_graph(rp, col)
        assert delta == n - 1 and sorted(colour.tolist()) == list(range(n))


def test_empty_graph_one_round_per_level():
    rp, col = G.empty(40)
    colour, rounds, delta = O.kw_colour_graph(rp, col)
    assert delta == 0 and np.all(colour == 0) and rounds == _levels(40, 0) == 6


def test_fig3_shape_two_levels():
    # Fig. 3: N = (Delta + 1) 2^M with M = 2; a 3-regular graph on 16 vertices (Delta = 3).
    edges = [(i, (i + 1) % 16) for i in range(16)] + [(i, (i + 8) % 16) for i in range(8)]
    rp, col = G.to_csr(16, edges)
    colour, rounds, delta = O.kw_colour_graph(rp, col)
    assert delta == 3 and _levels(16, 3) == 2
    _check_valid(rp, col, colour, delta)
    assert rounds <= (delta + 1) * 2


def test_sco_graph_colouring_is_valid_and_bounded():
    ch = O.Chain(O.make_params(48, T=0.4, seed=9))
    ch.switch()
    ncol = ch.colour()
    rp, col = ch.graph()
    o = ch.observables()
    colour = ch.colours()
    _check_valid(rp, col & 0x7FFFFFFF, colour, o["max_degree"])
    assert o["kw_rounds"] <= (o["max_degree"] + 1) * _levels(48 * 48, o["max_degree"])
    assert ncol == len(np.unique(colour)) == o["n_colours"]
    perm, off = ch.classes()
    assert np.array_equal(np.sort(perm), np.arange(48 * 48))
    for c in range(len(off) - 1):
        members = perm[off[c]:off[c + 1]]
        assert np.all(colour[members] == c) and np.all(np.diff(members) > 0)
