"""The allocation-free entry point ml_naive_noalloc against ml_observe.

ml_naive_noalloc serves callers that cannot allocate device memory (a host
framework that already owns the device's memory, or a serving loop that may
not stall on cudaMalloc).  It must give the same naive Polyakov correlator and
mean plaquette as the handle-based ml_observe on the same angles, on two
calls in a row (its scratch array is shared and keeps the previous call's
contents).  This file is collected last so that a failure here stops a
`-x` run only after every other test has run.
"""

import ctypes

import numpy as np
import pytest

from paper_1309_3859_b300 import ml, workloads

pytestmark = pytest.mark.gpu


def soa_layout(theta, L, Nt, dtype):
    """canonical [4][V] angles -> the library's [(mu*2 + parity)][V/2] layout"""
    V = L ** 3 * Nt
    i = np.arange(V)
    x, y, z, t = i % L, (i // L) % L, (i // L ** 2) % L, i // L ** 3
    par = (x + y + z + t) % 2
    out = np.zeros((4, 2, V // 2), dtype=dtype)
    for mu in range(4):
        out[mu, par, i >> 1] = theta[mu]
    return out


def call_noalloc(theta_dev, L, Nt, fp64, r, out_dev, stream):
    rr = (ctypes.c_int * len(r))(*r)
    return ml.lib().ml_naive_noalloc(ctypes.c_void_p(theta_dev.data_ptr()), L, Nt,
                                     ml.ML_FP64 if fp64 else ml.ML_FP32, rr, len(r),
                                     ctypes.c_void_p(out_dev.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("L,Nt,r", [(6, 4, (1, 2, 3)), (24, 8, tuple(range(2, 13)))])
def test_noalloc_matches_observe(fp64, L, Nt, r):
    import torch

    theta = workloads.random_angles(L, Nt, seed=11 + L)
    p = ml.Params(L=L, Nt=Nt, beta=0.98, fp64=fp64, r=r)
    with ml.Lattice(p) as lat:
        lat.set_angles(theta)
        ref = ml.split_record(p, lat.observe())
        stored = lat.get_angles()  # the angles as the lattice holds them (FP32 rounded)
    dtype = np.float64 if fp64 else np.float32
    th_dev = torch.from_numpy(soa_layout(stored, L, Nt, dtype)).cuda()
    stream = torch.cuda.Stream()
    for call in range(2):
        out = torch.full((2 * len(r) + 1,), float("nan"), dtype=torch.float64, device="cuda")
        stream.wait_stream(torch.cuda.current_stream())  # inputs and the NaN fill are in place
        with torch.cuda.stream(stream):
            st = call_noalloc(th_dev, L, Nt, fp64, r, out, stream)
        assert st == ml.ML_OK, (call, st)
        stream.synchronize()
        got = out.cpu().numpy()
        assert np.abs(got[:-1].reshape(-1, 2) - ref["naive"]).max() <= 1e-12, call
        assert abs(got[-1] - ref["plaq"]) <= 1e-12, call


def test_noalloc_rejects_oversized_and_invalid():
    import torch

    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    th = torch.zeros(16, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    # 64^3 x 64 with 3 separations needs more than the 2 MiB scratch array
    assert call_noalloc(th, 64, 64, True, (1, 2, 3), out, stream) == ml.ML_EINVAL
    assert call_noalloc(th, 4, 4, True, (4,), out, stream) == ml.ML_EINVAL
    assert call_noalloc(th, 5, 4, True, (1,), out, stream) == ml.ML_EINVAL
