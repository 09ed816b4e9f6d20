"""Batches of independent lattices (ml_batch_*): every lattice's records and
angles are bit-identical to the same parameters run alone, for both sweep
implementations and both precisions, with mixed sizes, couplings, seeds,
separations and probe sets."""

import numpy as np
import pytest

from paper_1309_3859_b300 import ml, workloads

pytestmark = pytest.mark.gpu


def mixed_params(fp64, n_sub=5, k_between=1, outer=False):
    base = dict(fp64=fp64, slab=2, n_sub=n_sub, k_between=k_between)
    if outer:
        base.update(outer_slab=4, n_sub_outer=2)
    nts = (8, 8, 4) if outer else (4, 6, 4)
    return [
        ml.Params(L=4, Nt=nts[0], beta=0.95, seed=11, r=(1, 2), rf=(2,), probes=((0, 0), (1, 0)), comp_mask=0x3F,
                  **base),
        ml.Params(L=6, Nt=nts[1], beta=0.97, seed=12, r=(1, 2, 3), rf=(2, 3), probes=((0, 0),), comp_mask=0x01,
                  **base),
        ml.Params(L=8, Nt=nts[2], beta=0.99, seed=13, r=(2, 4), rf=(4,), probes=((0, 0), (2, 1), (-1, 0)),
                  comp_mask=0x09, **base),
    ]


def run_alone(p, mode=None, n_therm=3, n_meas=2):
    with ml.Lattice(p) as lat:
        if mode is not None:
            lat.sweep_mode = mode
        lat.thermalize(n_therm)
        rec = lat.measure(n_meas)
        return rec, lat.get_angles()


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("mode", [ml.ML_SWEEP_PERSISTENT, ml.ML_SWEEP_PASSES, ml.ML_SWEEP_RESIDENT])
def test_batch_matches_alone(fp64, mode):
    ps = mixed_params(fp64, n_sub=20)
    alone = [run_alone(p, mode) for p in ps]
    with ml.Batch(ps) as b:
        b.sweep_mode = mode
        b.thermalize(3)
        recs = b.measure(2)
        angles = [b.get_angles(i) for i in range(len(ps))]
    for i in range(len(ps)):
        assert np.array_equal(recs[i], alone[i][0]), i
        assert np.array_equal(angles[i], alone[i][1]), i


@pytest.mark.parametrize("mode", [ml.ML_SWEEP_PERSISTENT, ml.ML_SWEEP_RESIDENT])
def test_batch_two_level_matches_alone(mode):
    ps = mixed_params(False, n_sub=3, outer=True)
    alone = [run_alone(p) for p in ps]
    with ml.Batch(ps) as b:
        b.sweep_mode = mode
        b.thermalize(3)
        recs = b.measure(2)
    for i in range(len(ps)):
        assert np.array_equal(recs[i], alone[i][0]), i


def test_batch_rejects_mixed_schedules():
    ps = mixed_params(False)
    ps[1].n_sub = 7
    with pytest.raises(ml.MLError):
        ml.Batch(ps)


def test_batch_mix_workload_runs():
    """64 lattices of the batched workload mix (L 12..24, Nt 4..12), one
    measurement each: finite records, per-lattice layouts."""
    mix = workloads.batch_mix(64)
    ps = [ml.Params(L=L, Nt=Nt, beta=beta, seed=seed, fp64=False, slab=2, n_sub=4, k_between=1,
                    r=tuple(range(1, L // 2 + 1)), rf=(L // 4,), probes=tuple((d, 0) for d in range(L // 4 + 1)),
                    comp_mask=workloads.COMP_EX) for (L, Nt, beta, seed) in mix]
    with ml.Batch(ps) as b:
        b.thermalize(2)
        recs = b.measure(1)
    for p, r in zip(ps, recs):
        s = ml.split_record(p, r)
        assert np.all(np.isfinite(r))
        assert 0.2 < float(s["plaq"][0]) < 0.9
