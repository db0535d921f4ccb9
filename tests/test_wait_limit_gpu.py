"""The failure path of the bounded device-side waits (grid barriers and neighbour waits of the
colouring and of the batched sweep), through the C ABI.

A wait limit of 0 ns makes a real wait give up: the kernel sets SCO_ETIMEOUT in the device
status word and returns (no trap, no fault, the GPU stays usable); the status becomes sticky,
so sco_sync and every later call of that context return it and the context does no more work.
A fresh context afterwards runs normally and still matches the oracle."""
import numpy as np
import pytest

import oracle as O
import paper_1503_03295_gb300 as sco

pytestmark = pytest.mark.gpu


def _status(call):
    try:
        call()
    except sco.ScoError as e:
        return e.status
    return sco.SCO_OK


def _device_still_works():
    g = sco.Lattice(sco.make_params(32, T=0.5, seed=2))
    o = O.Chain(O.make_params(32, T=0.5, seed=2))
    g.sweep(3)
    o.sweep(3)
    assert np.array_equal(g.spins(), o.spins())
    g.close()


@pytest.mark.parametrize("L", [256, 1024])  # per-level dataflow kernels; bucketed grid barriers
def test_colouring_wait_runs_out_and_the_context_refuses_work(L):
    lat = sco.Lattice(sco.make_params(L, T=0.3, seed=1))
    lat.switch()
    lat.set_wait_limit(0)
    assert _status(lambda: lat.colour()) == sco.SCO_ETIMEOUT
    assert _status(lat.sync) == sco.SCO_ETIMEOUT
    assert _status(lambda: lat.sweep(1)) == sco.SCO_ETIMEOUT
    assert _status(lat.switch) == sco.SCO_ETIMEOUT
    lat.close()
    _device_still_works()


def test_batched_wait_runs_out_and_the_batch_refuses_work():
    ps = sco.replica_params(L_list=(64, 128), n_T=2)
    b = sco.Batch(ps)
    b.run(1)
    b.set_wait_limit(0)
    assert _status(lambda: b.run(2)) == sco.SCO_ETIMEOUT
    assert _status(b.sync) == sco.SCO_ETIMEOUT
    assert _status(lambda: b.run(1)) == sco.SCO_ETIMEOUT
    b.close()
    _device_still_works()


def test_wait_limit_rejects_out_of_range():
    lat = sco.Lattice(sco.make_params(8, T=0.5, seed=1))
    assert _status(lambda: lat.set_wait_limit(3600 * 10**9 + 1)) == sco.SCO_EINVAL
    lat.set_wait_limit(2 * 10**9)
    lat.sweep(1)
    lat.close()
