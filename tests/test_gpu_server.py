"""Request server with continuous batching (ml_server_*, ml_submit, ml_poll).

* Each request's records are bit-identical to the same parameters run alone,
  with requests arriving while others run (different phases share ticks),
  mixed sizes, couplings, schedules and two-level requests.
* Multihit and Metropolis requests in the mix, bit-identical to alone.
* Size lanes: requests of different volumes tick in separate lanes (own
  streams and workers), records still as alone; one lane also works.
* Admission by HBM budget: requests queue until memory frees up, all finish,
  usage never exceeds the budget; a request larger than the budget fails with
  ML_ENOMEM; mismatched precision is rejected.
"""

import time

import numpy as np
import pytest

from paper_1309_3859_b300 import ml

pytestmark = pytest.mark.gpu


def job_params(i, fp64=False):
    base = dict(fp64=fp64, n_or=3)
    specs = [
        dict(L=4, Nt=4, beta=0.95, seed=101, slab=2, n_sub=5, k_between=1, r=(1, 2), rf=(2,),
             probes=((0, 0), (1, 0)), comp_mask=0x3F),
        dict(L=6, Nt=6, beta=0.97, seed=102, slab=2, n_sub=18, k_between=0, r=(1, 2, 3), rf=(3,),
             probes=((0, 0),), comp_mask=0x01),
        dict(L=8, Nt=8, beta=0.99, seed=103, slab=2, n_sub=3, outer_slab=4, n_sub_outer=2, k_between=2,
             r=(2, 4), rf=(4,), probes=((0, 0), (2, 1)), comp_mask=0x09),
        dict(L=6, Nt=4, beta=0.9, seed=104, slab=1, n_sub=4, k_between=1, r=(1,), rf=(1, 2),
             probes=((0, 0), (0, -1)), comp_mask=0x12),
    ]
    d = dict(specs[i % len(specs)])
    d["seed"] += 10 * (i // len(specs))
    d.update(base)
    return ml.Params(**d)


SCHED = [(3, 2), (0, 1), (2, 2), (4, 1), (1, 2), (5, 1)]  # (n_therm, n_meas)


def run_alone(p, n_therm, n_meas):
    with ml.Lattice(p) as lat:
        lat.thermalize(n_therm)
        return lat.measure(n_meas)


@pytest.mark.parametrize("fp64", [False, True])
def test_server_matches_alone(fp64):
    n = 6
    ps = [job_params(i, fp64) for i in range(n)]
    with ml.Server(budget_bytes=512 << 20, fp64=fp64) as srv:
        jobs = []
        for i in range(n):
            jobs.append(srv.submit(ps[i], *SCHED[i]))
            if i % 2 == 1:
                time.sleep(0.02)  # later requests arrive while earlier ones run
        results = [srv.wait(j, timeout_s=120) for j in jobs]
        st = srv.stats()
        assert st["completed"] == n and st["failed"] == 0 and st["used_bytes"] == 0
    for i in range(n):
        ref = run_alone(ps[i], *SCHED[i])
        assert np.array_equal(results[i], ref), i


def test_server_multihit_and_metropolis_requests_match_alone():
    """Requests with the analytic multihit (Section II.C) and with the
    Metropolis update, mixed with plain ones, give the records of the same
    parameters run alone."""
    ps = [job_params(i, False) for i in range(4)]
    ps[0].multihit = 1
    ps[1].multihit = 1
    ps[2].update, ps[2].metro_hits, ps[2].metro_width = ml.ML_UPDATE_METROPOLIS, 3, 1.4
    sched = [(2, 2), (1, 1), (2, 1), (0, 2)]
    with ml.Server(budget_bytes=256 << 20, fp64=False) as srv:
        jobs = [srv.submit(p, *sc) for p, sc in zip(ps, sched)]
        results = [srv.wait(j, timeout_s=120) for j in jobs]
    for i, p in enumerate(ps):
        assert np.array_equal(results[i], run_alone(p, *sched[i])), i


def test_server_budget_admission_and_limits():
    ps = [job_params(1, False) for _ in range(8)]
    for k, p in enumerate(ps):
        p.seed = 500 + k
    with ml.Server(budget_bytes=8 << 20, fp64=False) as srv:
        jobs = [srv.submit(p, 2, 1) for p in ps]
        peak_queue = 0
        while True:
            st = srv.stats()
            peak_queue = max(peak_queue, st["queued"])
            assert st["used_bytes"] <= st["budget_bytes"]
            if st["completed"] + st["failed"] == len(jobs):
                break
            time.sleep(0.001)
        assert st["failed"] == 0
        assert peak_queue > 0  # the budget held requests back
        for j in jobs:
            done, rec = srv.poll(j)
            assert done and np.all(np.isfinite(rec))
            t_sub, t_adm, t_done = srv.times(j)
            assert 0 <= t_sub <= t_adm <= t_done
        # a request that cannot fit even alone
        big = ml.Params(L=32, Nt=32, beta=1.0, fp64=False, slab=2, n_sub=2, r=(1,), rf=(2,),
                        probes=tuple((d, 0) for d in range(8)), comp_mask=0x3F)
        jb = srv.submit(big, 0, 1)
        with pytest.raises(ml.MLError) as exc:
            srv.wait(jb, timeout_s=60)
        assert exc.value.status == ml.ML_ENOMEM
        # precision must match the server's
        with pytest.raises(ml.MLError) as exc:
            srv.submit(job_params(0, fp64=True), 0, 1)
        assert exc.value.status == ml.ML_EINVAL


def test_server_lanes_match_alone():
    """Requests of different volumes go to different size lanes (below 2^16
    sites, below 2^18, above), which tick on their own streams at the same
    time; every request's records are still those of the same parameters run
    alone, and a lane of one lattice still advances small lattices by up to
    two sweeps per tick."""
    specs = [dict(L=4, Nt=4, n_sub=5, k_between=1), dict(L=16, Nt=16, n_sub=3, k_between=1),
             dict(L=24, Nt=20, n_sub=2, k_between=0), dict(L=6, Nt=8, n_sub=17, k_between=2),
             dict(L=16, Nt=12, n_sub=4, k_between=1)]
    ps = [ml.Params(beta=0.97, seed=700 + i, fp64=False, slab=2, r=(1, 2), rf=(2,), probes=((0, 0), (1, 0)),
                    comp_mask=0x09, **kw) for i, kw in enumerate(specs)]
    sched = [(5, 2), (3, 1), (1, 1), (4, 1), (2, 1)]
    with ml.Server(budget_bytes=2 << 30, fp64=False) as srv:
        jobs = []
        for p, sc in zip(ps, sched):
            jobs.append(srv.submit(p, *sc))
            time.sleep(0.01)
        results = [srv.wait(j, timeout_s=300) for j in jobs]
        st = srv.stats()
        assert st["completed"] == len(ps) and st["failed"] == 0 and st["used_bytes"] == 0
    for i, p in enumerate(ps):
        assert np.array_equal(results[i], run_alone(p, *sched[i])), i


def test_server_one_lane():
    """lanes = 1: every request in one tick loop, records as alone."""
    ps = [job_params(i, False) for i in range(3)]
    with ml.Server(budget_bytes=256 << 20, fp64=False, lanes=1) as srv:
        jobs = [srv.submit(p, 2, 1) for p in ps]
        results = [srv.wait(j, timeout_s=120) for j in jobs]
    for i, p in enumerate(ps):
        assert np.array_equal(results[i], run_alone(p, 2, 1)), i
