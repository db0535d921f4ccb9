"""The allocation-free colouring entry point (sco_kw_colour_static), through the C ABI.

It serves callers that cannot let a library allocate device memory while they run (their
device memory belongs to their own pool allocator, or a time-critical loop must not pay for
cudaMalloc/cudaFree).  Its output must equal the context path's (sco_colour): the same
colours bit for bit and the same max degree and t_R, on calls made back to back (the second
call reuses the scratch array that the first one left behind)."""
import ctypes as C

import numpy as np
import pytest

import paper_1503_03295_gb300 as sco

pytestmark = pytest.mark.gpu


def _reference(L, T, seed, J=0.0, D=1.0, variant=0):
    lat = sco.Lattice(sco.make_params(L, T=T, seed=seed, J=J, D=D, colour_variant=variant))
    lat.colour()
    rp, col = lat.graph()
    ref = lat.colours()
    obs = lat.observables()
    lat.close()
    return rp, col, ref, obs


def test_static_colouring_matches_sco_colour_on_consecutive_calls():
    import torch

    stream = torch.cuda.current_stream().cuda_stream
    cases = [(96, 0.4, 1, 0.0, 1.0, 0), (40, 0.8, 2, 1.0, 0.1, 0), (96, 0.4, 1, 0.0, 1.0, 1),
             (30, 1e12, 3, 0.0, 1.0, 0)]  # the last has no edges: palette of one colour
    for L, T, seed, J, D, variant in cases:
        rp, col, ref, obs = _reference(L, T, seed, J, D, variant)
        n = L * L
        d_rp = torch.from_numpy(rp.view(np.int32).copy()).cuda()
        # a graph without edges still passes a valid (one-entry) device buffer for col
        d_col = torch.from_numpy(col.view(np.int32).copy() if col.size else np.zeros(1, np.int32)).cuda()
        out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        for _ in range(2):  # two calls in a row on the same graph
            out.fill_(-1)
            delta, rounds = sco.kw_colour_static(d_rp.data_ptr(), d_col.data_ptr(), n,
                                                 out.data_ptr(), variant=variant, stream=stream)
            got = out.cpu().numpy().view(np.uint32)
            assert np.array_equal(got, ref)
            assert delta == obs["max_degree"] and rounds == obs["kw_rounds"]


def test_static_colouring_matches_the_oracle():
    # The same graphs coloured by the oracle's KW (Sec. 2.3.3), which runs the literal
    # synchronous rounds: colours and t_R must agree bit for bit.
    import oracle as O
    import torch

    stream = torch.cuda.current_stream().cuda_stream
    for L, T, seed, J, D, variant in [(64, 0.3, 5, 0.0, 1.0, 0), (48, 0.9, 6, 1.0, 0.1, 1)]:
        rp, col, _, _ = _reference(L, T, seed, J, D, variant)
        ref, ref_rounds, ref_delta = O.kw_colour_graph(rp.astype(np.int64), col, variant)
        n = L * L
        d_rp = torch.from_numpy(rp.view(np.int32).copy()).cuda()
        d_col = torch.from_numpy(col.view(np.int32).copy()).cuda()
        out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        delta, rounds = sco.kw_colour_static(d_rp.data_ptr(), d_col.data_ptr(), n,
                                             out.data_ptr(), variant=variant, stream=stream)
        assert np.array_equal(out.cpu().numpy(), ref)
        assert delta == ref_delta and rounds == ref_rounds


def test_static_colouring_at_its_maximum_size():
    # n = SCO_KW_STATIC_MAX_VERTICES exactly (an L = 1024 lattice at T = 0.4 D), where the
    # context path colours the upper KW levels with its bucketed kernel: same colours, max
    # degree and t_R, and no bounded wait runs out, on two calls in a row.
    import torch

    L = 1024
    assert L * L == sco.KW_STATIC_MAX_VERTICES
    stream = torch.cuda.current_stream().cuda_stream
    rp, col, ref, obs = _reference(L, 0.4, 1)
    n = L * L
    d_rp = torch.from_numpy(rp.view(np.int32).copy()).cuda()
    d_col = torch.from_numpy(col.view(np.int32).copy()).cuda()
    out = torch.empty((n,), dtype=torch.int32, device="cuda")
    for _ in range(2):
        out.fill_(-1)
        delta, rounds = sco.kw_colour_static(d_rp.data_ptr(), d_col.data_ptr(), n,
                                             out.data_ptr(), variant=0, stream=stream)
        assert np.array_equal(out.cpu().numpy().view(np.uint32), ref)
        assert delta == obs["max_degree"] and rounds == obs["kw_rounds"]


def test_static_colouring_rejects_oversize_without_device_work():
    lib = sco.load()
    d, r = C.c_int32(-7), C.c_int32(-7)
    st = lib.sco_kw_colour_static(C.c_void_p(16), C.c_void_p(16), sco.KW_STATIC_MAX_VERTICES + 1,
                                  0, C.c_void_p(16), C.byref(d), C.byref(r), None)
    assert st == sco.SCO_EINVAL and d.value == -7 and r.value == -7
