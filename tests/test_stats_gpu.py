"""Graph diagnostics (P_survive(r) of Fig. 5, P_IPC of Fig. 6, Delta R of Eq. (9)) and the
temperature change of the cooling protocol (Sec. 3.1), CUDA library against the oracle.

Counts are integers and must be equal; the per-shell and per-colour ratios are formed from equal
integers by one correctly rounded division each, so they must be equal too; the mean of Delta R
over the colours is a sum in another order (1e-14 relative)."""
import numpy as np
import pytest

import oracle as O
import paper_1503_03295_gb300 as sco

pytestmark = pytest.mark.gpu


def _same_stats(a, b):
    for k in ("n_pairs", "n_cross", "n_cells", "palette"):
        assert a[k] == b[k], k
    assert a["p_ipc"] == b["p_ipc"]
    for k in ("survived", "pairs"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["p_survive"], b["p_survive"], equal_nan=True)
    assert np.array_equal(a["delta_r"], b["delta_r"], equal_nan=True)
    assert a["delta_r_max"] == b["delta_r_max"]
    assert a["delta_r_weighted"] == b["delta_r_weighted"]
    assert abs(a["delta_r_mean"] - b["delta_r_mean"]) <= 1e-14 * max(abs(b["delta_r_mean"]), 1.0)


@pytest.mark.parametrize("L,T,J,D,cells,nb", [(64, 0.4, 0.0, 1.0, (4, 4), 32),
                                              (96, 4.5, 1.0, 0.1, (6, 8), 64),
                                              (50, 0.3, 0.0, 1.0, (50, 1), 4096),
                                              (33, 0.6, 0.0, 1.0, (1, 1), 1)])
def test_graph_stats_match_oracle(L, T, J, D, cells, nb):
    g = sco.Lattice(sco.make_params(L, T=T, J=J, D=D, seed=2))
    o = O.Chain(O.make_params(L, T=T, J=J, D=D, seed=2))
    g.sweep(3)
    o.sweep(3)
    _same_stats(g.graph_stats(*cells, nb), o.graph_stats(*cells, nb))


def test_graph_stats_need_a_colouring():
    g = sco.Lattice(sco.make_params(16, T=0.5, seed=1))
    with pytest.raises(sco.ScoError) as e:
        g.graph_stats(2, 2, 8)
    assert e.value.status == sco.SCO_ESTATE
    g.colour()
    with pytest.raises(sco.ScoError) as e:
        g.graph_stats(17, 1, 8)  # more cells than columns
    assert e.value.status == sco.SCO_EINVAL


@pytest.mark.parametrize("precision", [sco.FP64, sco.FP32_GUARDED])
def test_cooling_protocol_bit_exact(precision):
    # the paper's model (J = 1, D = 0.1) cooled in steps, n_sw = 5, the temperature changed
    # both at and between switch epochs: spins and accept bits equal the oracle's
    L = 32
    g = sco.Lattice(sco.make_params(L, T=1.25, J=1.0, D=0.1, seed=3, n_sw=5, precision=precision))
    o = O.Chain(O.make_params(L, T=1.25, J=1.0, D=0.1, seed=3, n_sw=5))
    for T, n in ((1.25, 5), (0.9, 7), (0.45, 6), (0.05, 9)):
        g.set_temperature(T)
        o.set_temperature(T)
        g.sweep(n)
        o.sweep(n)
        assert np.array_equal(g.accepts(), o.accepts()), T
        assert np.array_equal(g.spins(), o.spins()), T
        og, oo = g.observables(), o.observables()
        assert og["n_edges"] == oo["n_edges"] and og["kw_rounds"] == oo["kw_rounds"]
    with pytest.raises(sco.ScoError) as e:
        g.set_temperature(0.0)
    assert e.value.status == sco.SCO_EINVAL


def test_batched_cooling_matches_single_lattices():
    # three replicas of the paper's model cooled on different schedules, n_sw = 5, temperature
    # changes at multiples of n_sw: each replica equals a single lattice cooled the same way,
    # and replica 0 the oracle
    n_sw = 5
    ps = [sco.make_params(L, T=1.25, J=1.0, D=0.1, seed=10 + L, n_sw=n_sw,
                          precision=sco.FP32_GUARDED) for L in (24, 40, 17)]
    sched = [(1.25, 0.8, 0.45), (1.0, 0.5, 0.05), (0.9, 0.9, 0.3)]
    b = sco.Batch(ps)
    lats = [sco.Lattice(p) for p in ps]
    o = O.Chain(O.make_params(24, T=1.25, J=1.0, D=0.1, seed=34, n_sw=n_sw))
    for k in range(3):
        for r in range(3):
            b.set_temperature(r, sched[r][k])
            lats[r].set_temperature(sched[r][k])
        o.set_temperature(sched[0][k])
        b.run(2 * n_sw)
        for lat in lats:
            lat.sweep(2 * n_sw)
        o.sweep(2 * n_sw)
        for r in range(3):
            assert np.array_equal(b.spins(r), lats[r].spins()), (k, r)
            assert np.array_equal(b.accepts(r), lats[r].accepts()), (k, r)
        assert np.array_equal(b.spins(0), o.spins()), k
    b.run(2)
    with pytest.raises(sco.ScoError) as e:
        b.set_temperature(0, 0.5)  # step 32 is not a switch step
    assert e.value.status == sco.SCO_ESTATE
