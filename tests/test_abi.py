"""The C-ABI library builds for sm_103a, loads, and exports every declared entry point."""
import ctypes
import os
import re

import pytest

import paper_1503_03295_gb300 as sco
from paper_1503_03295_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(sco_\w+)\s*\(", txt))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("sco_init", "sco_switch", "sco_colour", "sco_sweep", "sco_observables",
              "sco_destroy", "sco_get_spins", "sco_set_spins", "sco_get_graph", "sco_sync"):
        assert n in names


def test_library_exports_every_declared_symbol():
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing
    assert sco.load() is not None


def test_status_strings():
    _build.build()
    assert sco.strerror(sco.SCO_OK) == "ok"
    assert "capacity" in sco.strerror(sco.SCO_ECAPACITY)


def test_invalid_parameters_rejected_before_any_device_work():
    _build.build()
    for bad in (dict(Lx=0), dict(Lx=4, T=0.0), dict(Lx=4, D=-1.0), dict(Lx=4, n_sw=0),
                dict(Lx=40000), dict(Lx=4, precision=7)):
        p = sco.make_params(**{"Lx": 4, **bad})
        with pytest.raises(sco.ScoError) as e:
            sco.Lattice(p)
        assert e.value.status == sco.SCO_EINVAL


def test_no_device_means_error_not_fallback():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    _build.build()
    with pytest.raises(sco.ScoError) as e:
        sco.Lattice(sco.make_params(8, T=0.5))
    assert e.value.status == sco.SCO_ECUDA


def test_batch_arguments_rejected_before_any_device_work():
    _build.build()
    good = sco.make_params(8, T=0.5)
    cases = [
        [],                                                          # no replica
        [good, sco.make_params(8, T=0.5, precision=sco.FP32_GUARDED)],  # mixed precision
        [good, sco.make_params(8, T=0.5, n_sw=2)],                   # mixed n_sw
        [good, sco.make_params(0, T=0.5)],                           # invalid replica
        [good] * 1025,                                               # too many replicas
    ]
    for ps in cases:
        with pytest.raises(sco.ScoError) as e:
            sco.Batch(ps)
        assert e.value.status == sco.SCO_EINVAL
