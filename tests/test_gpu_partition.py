"""Time-slab partition of one lattice (Section II.C: slabs are independent
given their frozen boundaries) against one process running ml_measure.

* One rank through the partition's steps (pass-by-pass k0 sweeps,
  ml_measure_inner, ml_measure_products): records bit-identical to
  ml_measure on the same chain.
* Two ranks (processes, gloo, both on cuda:0, host-staged exchanges; no
  kernel of one process waits on the other): records bit-identical to one
  process, and each rank's own time slices of the final configuration equal
  the single-process configuration's.  One level with a ring-buffer tail,
  two levels, FP32 and FP64.
"""

import os
import socket

import numpy as np
import pytest

from paper_1309_3859_b300 import ml

pytestmark = pytest.mark.gpu

CASES = {
    "one-level-fp32": dict(L=8, Nt=8, beta=0.98, seed=17, fp64=False, slab=2, n_sub=20, k_between=2, r=(1, 2, 3),
                           rf=(2, 3), probes=((0, 0), (1, 0), (0, 2)), comp_mask=0x3F),
    "two-level-fp64": dict(L=6, Nt=8, beta=0.95, seed=23, fp64=True, slab=2, n_sub=3, outer_slab=4, n_sub_outer=2,
                           k_between=1, r=(1, 2), rf=(2,), probes=((0, 0), (1, 0)), comp_mask=0x09),
    "one-level-fp64-multihit": dict(L=6, Nt=4, beta=0.9, seed=29, fp64=True, slab=2, n_sub=5, k_between=1,
                                    r=(1, 2, 3), rf=(2,), probes=((0, 0),), comp_mask=0x3F, multihit=1),
}
N_THERM, N_MEAS = 4, 2


def reference(kw):
    p = ml.Params(**kw)
    with ml.Lattice(p) as lat:
        lat.thermalize(N_THERM)
        recs = lat.measure(N_MEAS)
        return recs, lat.get_angles(), lat.sweep


@pytest.mark.parametrize("case", sorted(CASES))
def test_partition_one_rank_matches_measure(case):
    from paper_1309_3859_b300.partition import SlabPartition

    kw = CASES[case]
    ref, th_ref, n_ref = reference(kw)
    p = ml.Params(**kw)
    with ml.Lattice(p) as lat:
        lat.thermalize(N_THERM)
        got = SlabPartition(lat, p).measure(N_MEAS)
        th, n = lat.get_angles(), lat.sweep
    assert np.array_equal(got, ref)
    assert np.array_equal(th, th_ref) and n == n_ref


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, kw, out_dir):
    import torch
    import torch.distributed as dist

    from paper_1309_3859_b300.partition import SlabPartition

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        p = ml.Params(**kw)
        with ml.Lattice(p) as lat:
            lat.thermalize(N_THERM)  # the same whole-lattice chain on every rank
            part = SlabPartition(lat, p)
            recs = part.measure(N_MEAS)
            th = lat.get_angles()
            n = lat.sweep
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), recs=recs, th=th, n=n, t_lo=part.t_lo, t_hi=part.t_hi)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", sorted(CASES))
def test_partition_two_ranks_matches_one_process(case, tmp_path):
    import torch.multiprocessing as mp

    kw = CASES[case]
    mp.start_processes(_rank_main, args=(2, _free_port(), kw, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    ref, th_ref, n_ref = reference(kw)
    Ns = kw["L"] ** 3
    for rank in range(2):
        d = np.load(tmp_path / f"rank{rank}.npz")
        assert np.array_equal(d["recs"], ref), rank
        lo, hi = int(d["t_lo"]), int(d["t_hi"])
        own = slice(lo * Ns, hi * Ns)
        assert np.array_equal(d["th"][:, own], th_ref[:, own]), rank
        assert int(d["n"]) == n_ref


def test_partition_api_refusals():
    """ml_set_time_range validates its range (whole top-level slabs inside the
    lattice); with a partial range the whole-lattice schedules refuse
    (ML_ESTATE), as do products without a preceding inner phase; replay
    handles cannot be partitioned; (0, Nt) restores the whole lattice."""
    import torch

    p = ml.Params(**CASES["two-level-fp64"])  # Nt 8, outer slabs of 4
    with ml.Lattice(p) as lat:
        for lo, hi in [(0, 2), (2, 6), (-4, 4), (4, 12), (4, 4)]:
            with pytest.raises(ml.MLError) as e:
                lat.set_time_range(lo, hi)
            assert e.value.status == ml.ML_EINVAL, (lo, hi)
        lat.set_time_range(4, 8)
        for call in (lambda: lat.measure(1), lambda: lat.thermalize(1)):
            with pytest.raises(ml.MLError) as e:
                call()
            assert e.value.status == ml.ML_ESTATE
        rec = torch.zeros(lat.rec_len, dtype=torch.float64, device=lat.device)
        with pytest.raises(ml.MLError) as e:
            lat.measure_products(rec=rec)
        assert e.value.status == ml.ML_ESTATE
        lat.set_time_range(0, 8)
        assert np.all(np.isfinite(lat.measure(1)))
    q = ml.Params(**dict(CASES["one-level-fp32"], replay=1))
    with ml.Lattice(q) as lat:
        with pytest.raises(ml.MLError) as e:
            lat.set_time_range(0, 4)
        assert e.value.status == ml.ML_EINVAL
