"""Parity of the CUDA library (through the C ABI) with the oracle on the same seeded inputs.

Integer and decision outputs must be bit-exact: coupling table, initial spins, CSR graph of
surviving pairs, colours, t_R, colour classes (as sets), accept bits and spins after MC
steps (spins depend only on random words and accept bits).  Energies: within 1e-12
relative per spin (different summation order)."""
import numpy as np
import pytest

import oracle as O
import paper_1503_03295_gb300 as sco

pytestmark = pytest.mark.gpu

E_TOL = 1e-12


def _pair(L, Ly=None, **kw):
    prec = kw.pop("precision", sco.FP64)
    g = sco.Lattice(sco.make_params(L, Ly, precision=prec, **kw))
    o = O.Chain(O.make_params(L, Ly, **kw))
    return g, o


def _same_graph(g, o):
    rg, cg = g.graph()
    ro, co = o.graph()
    assert np.array_equal(rg.astype(np.int64), ro)
    assert np.array_equal(cg, co)


def _same_energy(a, b, N):
    assert abs(a - b) <= E_TOL * max(abs(a), abs(b), float(N))


@pytest.mark.parametrize("Lx,Ly", [(16, 16), (33, 17), (1, 9), (7, 1), (64, 64)])
def test_table_bit_exact(Lx, Ly):
    g = sco.Lattice(sco.make_params(Lx, Ly, T=0.5))
    t = g.table()
    r = O.table(Lx, Ly)
    assert np.array_equal(t["dx"], r["dx"]) and np.array_equal(t["dy"], r["dy"])
    assert np.array_equal(t["W"], r["W"])
    assert np.array_equal(t["Dc"], r["c"])  # D = 1: fl(D c) = c


@pytest.mark.parametrize("seed", [0, 5, 2**40 + 3])
def test_initial_spins_bit_exact(seed):
    g, o = _pair(48, T=0.5, seed=seed)
    assert np.array_equal(g.spins(), o.spins())


@pytest.mark.parametrize("L,T,J,seed", [(16, 0.5, 0.0, 0), (64, 0.3, 0.0, 1), (64, 1.2, 0.0, 2),
                                        (40, 0.6, 0.7, 3), (256, 0.6, 0.0, 1)])
def test_switch_graph_bit_exact(L, T, J, seed):
    g, o = _pair(L, T=T, J=J, seed=seed)
    g.switch()
    o.switch()
    _same_graph(g, o)
    og, oo = g.observables(), o.observables()
    assert og["n_edges"] == oo["n_edges"]
    assert og["max_degree"] == oo["max_degree"]
    assert og["max_degree_dipolar"] == oo["max_degree_dipolar"]


@pytest.mark.parametrize("L,T,variant", [(16, 0.5, 0), (64, 0.3, 0), (256, 0.6, 0), (64, 0.6, 1)])
def test_colouring_bit_exact(L, T, variant):
    g, o = _pair(L, T=T, seed=4, colour_variant=variant)
    ng = g.colour()
    no = o.colour()
    assert ng == no
    assert np.array_equal(g.colours().astype(np.int32), o.colours())
    og, oo = g.observables(), o.observables()
    assert og["kw_rounds"] == oo["kw_rounds"] and og["n_colours"] == oo["n_colours"]
    perm_g, off_g = g.classes()
    perm_o, off_o = o.classes()
    assert np.array_equal(off_g.astype(np.int64), off_o[:len(off_g)])
    # same members per class; inside a class: by tile of 2048 sites, then degree, then index
    rp, _ = g.graph()
    deg = np.diff(rp.astype(np.int64))
    for c in range(len(off_g) - 1):
        a, b = int(off_g[c]), int(off_g[c + 1])
        mine = perm_g[a:b].astype(np.int64)
        assert np.array_equal(np.sort(mine), perm_o[a:b])
        dk = 64
        while dk > 1 and (len(off_g) - 1) * dk > 8192:
            dk //= 2
        tiles, bins = mine // 2048, np.minimum(deg[mine], dk - 1)
        order = np.lexsort((mine, bins, tiles))
        assert np.array_equal(order, np.arange(len(mine)))


@pytest.mark.parametrize("L,T,J,n", [(16, 0.5, 0.0, 200), (64, 0.3, 0.0, 20), (64, 1.2, 0.0, 20),
                                     (32, 0.8, 1.0, 20), (32, 0.08, 0.0, 30)])
def test_trajectory_bit_exact(L, T, J, n):
    """FP64 form against the oracle step by step; T = 0.08 D (beta D = 12.5) drives the decision's
    products below 2^-600 (their renormalisation) and its exponentials over a wide range."""
    g, o = _pair(L, T=T, J=J, D=1.0 if J == 0 else 0.1, seed=7)
    for k in range(n):
        g.sweep(1)
        o.sweep(1)
        if k % max(1, n // 5) == 0 or k == n - 1:
            assert np.array_equal(g.accepts(), o.accepts()), k
            assert np.array_equal(g.spins(), o.spins()), k
    _same_graph(g, o)
    og, oo = g.observables(full=True), o.observables(full=True)
    for key in ("e_switched", "e_exchange", "e_full"):
        _same_energy(og[key], oo[key], g.N)
    for key in ("mx", "my", "mz", "m_abs", "m_phi"):
        assert abs(og[key] - oo[key]) < 1e-13
    assert og["sweeps_done"] == oo["sweeps_done"] == n


@pytest.mark.parametrize("T", [0.3, 0.6, 1.2])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_l256_first_50_sweeps(T, seed):
    """The L = 256 workload, every (T, seed) pair of it: accept bits and spins bit-exact after
    sweeps 1, 10 and 50, energy within 1e-12 relative."""
    g, o = _pair(256, T=T, seed=seed)
    done = 0
    for upto in (1, 10, 50):
        g.sweep(upto - done)
        o.sweep(upto - done)
        done = upto
        assert np.array_equal(g.accepts(), o.accepts()), upto
        assert np.array_equal(g.spins(), o.spins()), upto
    _same_energy(g.observables()["e_switched"], o.observables()["e_switched"], g.N)


@pytest.mark.parametrize("T", [0.4, 0.8])
def test_fp32_guarded_matches_fp64_and_oracle(T):
    L = 96
    g64 = sco.Lattice(sco.make_params(L, T=T, seed=1))
    g32 = sco.Lattice(sco.make_params(L, T=T, seed=1, precision=sco.FP32_GUARDED))
    o = O.Chain(O.make_params(L, T=T, seed=1))
    g64.sweep(15)
    g32.sweep(15)
    o.sweep(15)
    s = o.spins()
    assert np.array_equal(g64.spins(), s)
    assert np.array_equal(g32.spins(), s)
    e32, e64 = g32.observables(), g64.observables()
    assert abs(e32["e_switched"] - e64["e_switched"]) <= 1e-6 * abs(e64["e_switched"])
    assert e32["guard_hits_fp32"] > 0  # the FP32 screen did defer some decisions


def test_edge_cases_tiny_lattices():
    for (Lx, Ly) in [(1, 1), (2, 1), (1, 2), (3, 1)]:
        g, o = _pair(Lx, Ly, T=0.3, seed=9)
        g.sweep(5)
        o.sweep(5)
        assert np.array_equal(g.spins(), o.spins())
        assert g.observables()["n_colours"] == o.observables()["n_colours"]


def test_infinite_temperature_and_pure_exchange():
    g, o = _pair(20, T=1e12, seed=2)
    g.sweep(2)
    o.sweep(2)
    assert np.array_equal(g.spins(), o.spins()) and np.all(g.accepts() == 1)
    og, oo = g.observables(), o.observables()
    assert og["n_edges"] == 0 and og["max_degree"] == 0
    assert og["kw_rounds"] == oo["kw_rounds"] and np.all(g.colours() == 0)
    g, o = _pair(12, T=0.7, J=1.0, D=0.0, seed=3)
    g.sweep(4)
    o.sweep(4)
    assert np.array_equal(g.spins(), o.spins())
    _same_graph(g, o)


def test_checkpoint_resume_bit_exact():
    for n_sw in (1, 3):
        p = dict(T=0.5, seed=11, n_sw=n_sw)
        a = sco.Lattice(sco.make_params(32, **p))
        a.sweep(10)
        ref = a.spins()
        b = sco.Lattice(sco.make_params(32, **p))
        b.sweep(4)
        blob = b.get_state()
        c = sco.Lattice(sco.make_params(32, **p))
        c.set_state(blob)
        c.sweep(6)
        assert np.array_equal(c.spins(), ref)
        o = O.Chain(O.make_params(32, **p))
        o.sweep(10)
        assert np.array_equal(o.spins(), ref)


@pytest.mark.slow
def test_full_size_first_sweep_L2304():
    """The workload size of the throughput benchmark: L = 2304, T = 0.6 D, seed 0, in both
    forms the benchmark times (FP64 and FP32-guarded), against two oracle MC steps."""
    g, o = _pair(2304, T=0.6, seed=0)
    t = g.table()
    r = O.table(2304)
    idx = np.random.default_rng(0).integers(0, len(r["W"]), 200000)
    assert np.array_equal(t["W"][idx], r["W"][idx]) and np.array_equal(t["dx"][idx], r["dx"][idx])
    del t, r
    g.sweep(1)
    o.sweep(1)
    _same_graph(g, o)
    assert np.array_equal(g.colours().astype(np.int32), o.colours())
    assert np.array_equal(g.spins(), o.spins())
    og, oo = g.observables(), o.observables()
    assert og["kw_rounds"] == oo["kw_rounds"]
    assert og["max_degree_dipolar"] == oo["max_degree_dipolar"]
    _same_energy(og["e_switched"], oo["e_switched"], g.N)
    # the graph diagnostics at full size, for the processor counts of Fig. 6
    for cx, cy in ((6, 8), (16, 18)):
        a, b = g.graph_stats(cx, cy, 64), o.graph_stats(cx, cy, 64)
        assert a["n_cross"] == b["n_cross"] and np.array_equal(a["survived"], b["survived"])
        assert np.array_equal(a["pairs"], b["pairs"])
        assert a["delta_r_weighted"] == b["delta_r_weighted"]
        assert np.array_equal(a["delta_r"], b["delta_r"], equal_nan=True)
    # a second MC step (a new switch, the FP64 pair cache filled again)
    g.sweep(1)
    o.sweep(1)
    assert np.array_equal(g.accepts(), o.accepts())
    assert np.array_equal(g.spins(), o.spins())
    og, oo = g.observables(), o.observables()
    assert og["kw_rounds"] == oo["kw_rounds"]
    _same_energy(og["e_switched"], oo["e_switched"], g.N)
    g.close()
    g32 = sco.Lattice(sco.make_params(2304, T=0.6, seed=0, precision=sco.FP32_GUARDED))
    g32.sweep(2)
    _same_graph(g32, o)
    assert np.array_equal(g32.colours().astype(np.int32), o.colours())
    assert np.array_equal(g32.spins(), o.spins())
    assert np.array_equal(g32.accepts(), o.accepts())
    o32 = g32.observables()
    assert o32["kw_rounds"] == oo["kw_rounds"]
    assert abs(o32["e_switched"] - og["e_switched"]) <= 1e-6 * abs(og["e_switched"])


@pytest.mark.slow
@pytest.mark.parametrize("T", [0.4, 0.8])
def test_fp32_guarded_L1024(T):
    """The precision workload's size: L = 1024, FP32-guarded against FP64 on the same seed
    (identical decisions, energy within 1e-6 relative) and both against the oracle."""
    L, n = 1024, 3
    g64 = sco.Lattice(sco.make_params(L, T=T, seed=1))
    g32 = sco.Lattice(sco.make_params(L, T=T, seed=1, precision=sco.FP32_GUARDED))
    o = O.Chain(O.make_params(L, T=T, seed=1))
    g64.sweep(n)
    g32.sweep(n)
    o.sweep(n)
    s = o.spins()
    assert np.array_equal(g64.spins(), s)
    assert np.array_equal(g32.spins(), s)
    assert np.array_equal(g32.accepts(), o.accepts())
    e32, e64, eo = g32.observables(), g64.observables(), o.observables()
    assert abs(e32["e_switched"] - e64["e_switched"]) <= 1e-6 * abs(e64["e_switched"])
    _same_energy(e64["e_switched"], eo["e_switched"], g64.N)
    assert e32["kw_rounds"] == eo["kw_rounds"] and e32["n_colours"] == eo["n_colours"]


def test_library_expm1_within_its_bound():
    """The FP64 decisions take expm1 from the library's own branch-free implementation with a
    stated relative error bound of 2^-42 (carried in their error bounds); check it against
    double-double on 16M points of [-50, 0.35] (range ends, the -40 cut, reduction boundaries
    included)."""
    err, diff = sco.selftest_expm1(1 << 24, seed=3)
    assert err < 2.0 ** -42
    assert diff < 2.0 ** -42
    # the degree-6 variant of the sweep decisions, stated bound 2^-31
    err, diff = sco.selftest_expm1(1 << 24, seed=4, degree=6)
    assert err < 2.0 ** -31
    assert diff < 2.0 ** -31


def test_library_log_within_its_bound():
    """The FP64 candidate search of the switch takes log from the library's own table-driven
    implementation with a stated relative error bound of 2^-49 (carried in its margin); check it
    against double-double on 16M points of (0, 1] (all octaves, values just below 1, the
    reduction and table boundaries)."""
    err, diff = sco.selftest_log(1 << 24, seed=5)
    assert err < 2.0 ** -49
    assert diff < 2.0 ** -49


def test_fp64_pair_cache_paths_bit_exact():
    """The FP64 form carries the pair terms of one MC step to the next on the same graph
    (n_sw > 1), rebuilds them after spins were set from outside, and starts from the switch's
    values after every switch: with exchange bonds in the graph, every path keeps the accept bits
    and spins equal to the oracle's."""
    L = 40
    p = dict(T=0.35, J=0.5, D=1.0, seed=13, n_sw=4)
    g, o = _pair(L, **p)
    rng = np.random.default_rng(3)
    plan = [5, "same", 3, "new", 6, 4]
    for step in plan:
        if step == "same":  # set_spins with the current spins: cached terms rebuilt, same values
            x = g.spins()
            g.set_spins(x)
            o.set_spins(x)
            continue
        if step == "new":  # fresh spins in the middle of an epoch: the graph stays
            v = rng.normal(size=(L * L, 3))
            v /= np.linalg.norm(v, axis=1, keepdims=True)
            x = v.T.reshape(-1).copy()
            g.set_spins(x)
            o.set_spins(x)
            continue
        for _ in range(step):
            g.sweep(1)
            o.sweep(1)
            assert np.array_equal(g.accepts(), o.accepts())
        assert np.array_equal(g.spins(), o.spins())
    og, oo = g.observables(), o.observables()
    _same_energy(og["e_switched"], oo["e_switched"], g.N)


def test_fp64_pair_cache_carry_thread_path():
    """The carried pair terms through the one-thread-per-site sweep (classes above 4096 sites):
    L = 384 with n_sw = 4, two epochs, accept bits and spins equal to the oracle's."""
    g, o = _pair(384, T=0.6, seed=21, n_sw=4)
    for k in range(8):
        g.sweep(1)
        o.sweep(1)
        assert np.array_equal(g.accepts(), o.accepts()), k
    assert np.array_equal(g.spins(), o.spins())

