"""Launch timeline of the measurement schedule (ml_timeline_enable,
ml_timeline_read): the marks come in begin/end pairs in the order Algorithm
1 enqueues them (full sweeps, then the sub-update groups of each ring buffer
on the main stream; a fold per ring buffer and the products on the
accumulation stream), their times increase along each stream, the capacity
bounds them, and recording them leaves the records bit-identical."""

import numpy as np
import pytest

from paper_1309_3859_b300 import ml

pytestmark = pytest.mark.gpu

KW = dict(L=8, Nt=8, beta=0.95, seed=5, fp64=False, slab=2, n_sub=37, k_between=2, r=(1, 2), rf=(2,),
          probes=((0, 0), (1, 0)), comp_mask=0x3F)
MAIN = {ml.ML_TL_FULL_BEGIN, ml.ML_TL_FULL_END, ml.ML_TL_SUB_BEGIN, ml.ML_TL_SUB_END}


def run(mode, timeline):
    p = ml.Params(**KW)
    with ml.Lattice(p) as lat:
        if mode is not None:
            lat.sweep_mode = mode
        lat.thermalize(2)
        if timeline:
            lat.timeline_enable(timeline)
        recs = lat.measure(2)
        marks = lat.timeline() if timeline else []
        return recs, marks, lat.batch_slots


@pytest.mark.parametrize("mode", [ml.ML_SWEEP_PERSISTENT, ml.ML_SWEEP_PASSES, ml.ML_SWEEP_RESIDENT])
def test_timeline_marks(mode):
    ref, _, _ = run(mode, 0)
    recs, marks, nB = run(mode, 1024)
    assert np.array_equal(recs, ref)
    nbuf = -(-KW["n_sub"] // nB)
    tags = [t for t, _ in marks]
    main = [t for t in tags if t in MAIN]
    side = [t for t in tags if t not in MAIN]
    per_meas_main = [ml.ML_TL_FULL_BEGIN, ml.ML_TL_FULL_END] + [ml.ML_TL_SUB_BEGIN, ml.ML_TL_SUB_END] * nbuf
    assert main == per_meas_main * 2
    per_meas_side = [ml.ML_TL_FOLD_BEGIN, ml.ML_TL_FOLD_END] * nbuf + [ml.ML_TL_PROD_BEGIN, ml.ML_TL_PROD_END]
    assert side == per_meas_side * 2
    assert marks[0][1] == 0.0
    for stream in (MAIN, None):
        times = [ms for t, ms in marks if (t in MAIN) == (stream is not None)]
        assert all(b >= a for a, b in zip(times, times[1:]))
    assert all(ms >= 0.0 for _, ms in marks)


def test_timeline_capacity_and_off():
    p = ml.Params(**KW)
    with ml.Lattice(p) as lat:
        lat.thermalize(1)
        lat.timeline_enable(5)
        lat.measure(1)
        assert len(lat.timeline()) == 5
        lat.measure(1)  # the capacity stays, the marks were discarded
        assert len(lat.timeline()) == 5
        lat.timeline_enable(0)
        lat.measure(1)
        assert lat.timeline() == []
        with pytest.raises(ml.MLError) as e:
            lat.timeline_enable(-1)
        assert e.value.status == ml.ML_EINVAL


def test_resident_profile():
    """The timed cluster-resident launch (ml_resident_profile): every phase
    takes time, the passes and records account for most of the launch, the
    chain is unchanged (the launch runs on the timing copy), and handles whose
    sub-updates are not cluster-resident are refused."""
    p = ml.Params(**KW)
    with ml.Lattice(p) as lat:
        lat.sweep_mode = ml.ML_SWEEP_RESIDENT
        lat.thermalize(1)
        before = lat.get_angles()
        prof = lat.resident_profile()
        assert np.array_equal(lat.get_angles(), before)
        assert prof["sub_updates"] == lat.batch_slots and prof["ctas"] > 0
        for k in ("update_heatbath_t", "update_heatbath_s", "update_overrelax_t", "update_overrelax_s",
                  "exchange_heatbath_t", "exchange_overrelax_s", "record", "setup", "write_back"):
            assert prof[k] > 0, k
        n_or = p.n_or
        per_sub = (2 * (prof["update_heatbath_t"] + prof["exchange_heatbath_t"])
                   + 6 * (prof["update_heatbath_s"] + prof["exchange_heatbath_s"])
                   + 2 * n_or * (prof["update_overrelax_t"] + prof["exchange_overrelax_t"])
                   + 6 * n_or * (prof["update_overrelax_s"] + prof["exchange_overrelax_s"]) + prof["record"])
        parts = per_sub * prof["sub_updates"] + prof["setup"] + prof["write_back"]
        assert 0.8 * prof["launch"] < parts <= 1.01 * prof["launch"]
        ref = lat.measure(1)
    with ml.Lattice(p) as lat:
        lat.sweep_mode = ml.ML_SWEEP_RESIDENT
        lat.thermalize(1)
        assert np.array_equal(lat.measure(1), ref)
        lat.sweep_mode = ml.ML_SWEEP_PASSES
        with pytest.raises(ml.MLError) as e:
            lat.resident_profile()
        assert e.value.status == ml.ML_EINVAL
