"""Batched replicas (sco_batch_*) through the C ABI.

Replica r of a batch must follow exactly the trajectory of a single lattice created with the
same parameters: same switched graph, colours, t_R, accept bits and spins (bit for bit), and
observables up to summation order.  That must hold whatever the tuning (graph replay or
direct launches, grid sizes, steps per graph) and across replans (device buffers grown after
a step that would have overflowed them).  A few replicas are also checked against the
oracle directly."""
import numpy as np
import pytest

import oracle as O
import paper_1503_03295_gb300 as sco

pytestmark = pytest.mark.gpu

E_TOL = 1e-12


def _single(p, n):
    lat = sco.Lattice(p)
    lat.sweep(n)
    return lat


def _mixed(precision):
    return [sco.make_params(16, T=0.5, seed=0, precision=precision),
            sco.make_params(33, 17, T=0.3, seed=5, precision=precision),
            sco.make_params(1, 9, T=0.7, seed=2, precision=precision),
            sco.make_params(64, T=1.2, seed=3, precision=precision),
            sco.make_params(40, T=0.6, J=1.0, D=0.1, seed=4, precision=precision),
            sco.make_params(48, T=0.4, seed=6, precision=precision, colour_variant=1),
            sco.make_params(7, 1, T=0.3, seed=7, precision=precision),
            sco.make_params(20, T=1e12, seed=8, precision=precision)]


def _same_replica(b, r, lat, n_steps):
    assert np.array_equal(b.spins(r), lat.spins()), r
    assert np.array_equal(b.accepts(r), lat.accepts()), r
    rg, cg = b.graph(r)
    ro, co = lat.graph()
    assert np.array_equal(rg, ro) and np.array_equal(cg, co), r
    assert np.array_equal(b.colours(r), lat.colours()), r
    ob, ol = b.observables(r), lat.observables()
    for k in ("n_edges", "max_degree", "max_degree_dipolar", "n_colours", "kw_rounds"):
        assert ob[k] == ol[k], (r, k, ob[k], ol[k])
    assert ob["sweeps_done"] == ol["sweeps_done"] == n_steps
    for k in ("e_switched", "e_exchange"):
        assert abs(ob[k] - ol[k]) <= E_TOL * max(abs(ol[k]), lat.N), (r, k)


@pytest.mark.parametrize("precision", [sco.FP64, sco.FP32_GUARDED])
def test_batch_matches_single_lattices(precision):
    ps = _mixed(precision)
    n = 6
    with sco.Batch(ps) as b:
        b.run(n)
        assert b.info()["steps_done"] == n
        for r, p in enumerate(ps):
            lat = _single(p, n)
            _same_replica(b, r, lat, n)
            lat.close()


def test_batch_matches_oracle():
    ps = [sco.make_params(16, T=0.5, seed=0), sco.make_params(24, 13, T=0.35, seed=9),
          sco.make_params(12, T=0.7, J=1.0, D=0.1, seed=3)]
    n = 10
    with sco.Batch(ps) as b:
        b.run(n)
        for r, p in enumerate(ps):
            o = O.Chain(O.make_params(p.Lx, p.Ly, T=p.T, J=p.J, D=p.D, seed=p.seed))
            o.sweep(n)
            assert np.array_equal(b.spins(r), o.spins()), r
            assert np.array_equal(b.accepts(r), o.accepts()), r


def test_results_do_not_depend_on_tuning():
    ps = _mixed(sco.FP32_GUARDED)[:6]
    n = 9
    ref = sco.Batch(ps)
    ref.set_tuning(steps_per_graph=1, sweep_blocks_per_sm=1, kw_blocks_per_sm=1, use_graph=0,
                   kw_schedule=1, kw_low=0)
    ref.run(n)
    want = [ref.spins(r) for r in range(len(ps))]
    want_c = [ref.colours(r) for r in range(len(ps))]
    want_t = [ref.observables(r)["kw_rounds"] for r in range(len(ps))]
    for t in (dict(steps_per_graph=4, sweep_blocks_per_sm=2, kw_blocks_per_sm=2, use_graph=1),
              dict(steps_per_graph=3, sweep_blocks_per_sm=6, kw_blocks_per_sm=4, use_graph=1,
                   kw_low=2),
              dict(steps_per_graph=1, sweep_blocks_per_sm=3, kw_blocks_per_sm=1, use_graph=0,
                   kw_low=0),
              dict(steps_per_graph=2, sweep_blocks_per_sm=4, kw_blocks_per_sm=2, use_graph=1,
                   kw_schedule=1),
              dict(steps_per_graph=2, sweep_blocks_per_sm=2, kw_blocks_per_sm=1, use_graph=1,
                   kw_schedule=1, kw_low=2),
              dict(steps_per_graph=2, sweep_blocks_per_sm=2, kw_blocks_per_sm=2, use_graph=1,
                   kw_low_group=4096),
              dict(steps_per_graph=1, sweep_blocks_per_sm=2, kw_blocks_per_sm=2, use_graph=0,
                   kw_schedule=1, kw_low_group=1024)):
        with sco.Batch(ps) as b:
            b.set_tuning(**t)
            b.run(4)
            b.run(n - 4)
            for r in range(len(ps)):
                assert np.array_equal(b.spins(r), want[r]), (t, r)
                assert np.array_equal(b.colours(r), want_c[r]), (t, r)
                assert b.observables(r)["kw_rounds"] == want_t[r], (t, r)
    with sco.Batch(ps) as b:
        chosen = b.autotune(trial_steps=1)  # the trial steps are real MC steps
        assert chosen["steps_per_graph"] >= 1
        b.run(3)
        total = b.info()["steps_done"]
        assert total > n
        ref.run(total - n)
        for r in range(len(ps)):
            assert np.array_equal(b.spins(r), ref.spins(r)), ("autotuned", chosen, r)
    ref.close()


def test_replan_on_overflowing_graph():
    """Very low T: CSR entries above the initial 24 per site, half-degrees above the 32
    per-site slots (overflow list larger than its initial size) and a palette above 256
    colours, all in one step; the step is repeated after the buffers grow."""
    ps = [sco.make_params(32, T=0.004, seed=1), sco.make_params(16, T=0.5, seed=2)]
    with sco.Batch(ps) as b:
        b.run(2)
        info = b.info()
        assert info["replans"] >= 1 and info["steps_done"] == 2
        assert b.observables(0)["max_degree"] > 255
        for r, p in enumerate(ps):
            lat = _single(p, 2)
            _same_replica(b, r, lat, 2)
            lat.close()


def test_n_sw_epochs():
    ps = [sco.make_params(24, T=0.5, seed=1, n_sw=3), sco.make_params(40, 8, T=0.9, seed=2, n_sw=3)]
    with sco.Batch(ps) as b:
        b.set_tuning(steps_per_graph=2, sweep_blocks_per_sm=2, kw_blocks_per_sm=2, use_graph=1)
        b.run(7)
        for r, p in enumerate(ps):
            lat = _single(p, 7)
            assert np.array_equal(b.spins(r), lat.spins()), r
            lat.close()


def test_set_spins_roundtrip_and_errors():
    ps = [sco.make_params(8, T=0.5, seed=1), sco.make_params(12, T=0.5, seed=2)]
    with sco.Batch(ps) as b:
        x = b.spins(1)
        b.set_spins(1, x[::-1].copy())
        assert np.array_equal(b.spins(1), x[::-1])
        with pytest.raises(sco.ScoError) as e:
            b.observables(2)  # replica index out of range
        assert e.value.status == sco.SCO_EINVAL
        with pytest.raises(sco.ScoError) as e:
            b.graph(0)  # no graph before the first step
        assert e.value.status == sco.SCO_ESTATE


@pytest.mark.slow
def test_batched_workload_64_replicas():
    """The batched workload itself: 64 replicas (L in {64, 128, 256, 512} x 16 temperatures in
    [0.2, 1.5] D), FP32-guarded, autotuned; after its steps, sampled replicas of every size
    (lowest and highest T) equal their single-lattice runs, and one small one the oracle."""
    ps = sco.replica_params()
    with sco.Batch(ps) as b:
        b.autotune(trial_steps=1)
        b.run(2)
        n = b.info()["steps_done"]
        for r in (0, 15, 16, 31, 32, 47, 48, 63):
            lat = _single(ps[r], n)
            _same_replica(b, r, lat, n)
            lat.close()
        # against the oracle directly: a small replica, and both ends of the largest size
        # (replica 48: L = 512 at T = 0.2 D, mean degree about 37, the most work per site;
        # replica 63: L = 512 at T = 1.5 D): spins, accept bits of the last step, colours, t_R
        for r in (3, 48, 63):
            p = ps[r]
            o = O.Chain(O.make_params(p.Lx, p.Ly, T=p.T, J=p.J, D=p.D, seed=p.seed))
            o.sweep(n)
            assert np.array_equal(b.spins(r), o.spins()), r
            assert np.array_equal(b.accepts(r), o.accepts()), r
            assert np.array_equal(b.colours(r).astype(np.int32), o.colours()), r
            assert b.observables(r)["kw_rounds"] == o.observables()["kw_rounds"], r
            o.close()
