"""Host-side checks of the C ABI that need no GPU.

* libml.so builds, loads and exports every function include/ml.h declares.
* ml_record_len agrees with the oracle's record layout.
* Invalid parameter sets are rejected with ML_EINVAL before any device work.
"""

import ctypes
import os
import re

import pytest

import oracle
from paper_1309_3859_b300 import ml

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ml.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ml_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("ml_create", "ml_thermalize", "ml_measure", "ml_destroy", "ml_record_len", "ml_error_string"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = ml.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
        assert name in ml.SIGNATURES, name


def test_error_strings():
    L = ml.lib()
    for st in range(0, -8, -1):
        assert L.ml_error_string(st)
    assert L.ml_error_string(ml.ML_EINVAL) == b"invalid argument"


@pytest.mark.parametrize("nr,nrf,npb", [(1, 0, 0), (4, 2, 4), (11, 11, 9), (23, 3, 13)])
def test_record_len_matches_oracle(nr, nrf, npb):
    r = tuple(range(1, nr + 1))
    rf = tuple(range(1, nrf + 1))
    probes = tuple((d, 0) for d in range(npb))
    p = ml.Params(L=64, Nt=4, beta=1.0, r=r, rf=rf, probes=probes, comp_mask=0x3F)
    po = oracle.Params(L=64, Nt=4, beta=1.0, r=r, rf=rf, probes=probes, comp_mask=0x3F)
    assert ml.record_len(p) == oracle.record_len(po)


BAD = [
    dict(L=5), dict(Nt=3), dict(L=0), dict(beta=-0.1), dict(slab=3), dict(n_sub=0), dict(outer_slab=3),
    dict(outer_slab=8, n_sub_outer=1, Nt=4), dict(outer_slab=4, n_sub_outer=0), dict(outer_slab=2, n_sub_outer=1),
    dict(r=(0,)), dict(r=(4,)), dict(r=()), dict(rf=(5,)), dict(probes=((4, 0),)), dict(probes=((0, -4),)),
    dict(comp_mask=64), dict(k_between=-1), dict(n_or=-1), dict(Nt=256, slab=2),
]


@pytest.mark.parametrize("bad", BAD)
def test_create_rejects_invalid_parameters(bad):
    kw = dict(L=4, Nt=4, beta=1.0, slab=2, n_sub=1, r=(1,), rf=(1,), probes=((0, 0),), comp_mask=1)
    kw.update(bad)
    p = ml.Params(**kw)
    h = ctypes.c_void_p()
    st = ml.lib().ml_create(ctypes.byref(p.c()), None, None, ctypes.byref(h))
    assert st == ml.ML_EINVAL
    assert not h.value


def test_null_arguments_rejected():
    L = ml.lib()
    assert L.ml_destroy(None) == ml.ML_EINVAL
    assert L.ml_thermalize(None, 1) == ml.ML_EINVAL
    assert L.ml_measure(None, 1, None, 0) == ml.ML_EINVAL
    assert L.ml_record_len(None, None) == ml.ML_EINVAL
    assert L.ml_philox(None, None, 0, None) == ml.ML_EINVAL
