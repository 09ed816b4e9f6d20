"""GPU chains against theory and against the oracle's chain, statistically.

* Strong coupling: <cos theta_p> = I1(beta)/I0(beta) + O(u^5), FP64 and FP32,
  heatbath and Metropolis chains.
* A Metropolis chain (Section II's update) and a heatbath chain sample the
  same ensemble: plaquette and P(r) agree within errors.
* FP32 and FP64 GPU chains against an independent FP64 oracle chain:
  plaquette, P(r), field insertions and vacuum within 3 combined standard
  errors (jackknife over measurements).
* Multilevel P(r) against the naive estimator on the small workload.
* Multihit P(r) against the plain estimator on the same chain (paired
  differences) and its smaller error.
* beta = 0: zero means.
* Gauge covariance of one GPU heatbath sweep.
All seeds are fixed and the GPU reductions run in a fixed order, so each of
these tests is deterministic.
"""

import numpy as np
import pytest
import scipy.special as sp

import oracle
from paper_1309_3859_b300 import ml, workloads
from paper_1309_3859_b300.stats import jackknife

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi


@pytest.mark.parametrize("update", [ml.ML_UPDATE_HEATBATH, ml.ML_UPDATE_METROPOLIS])
@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("beta", [0.1, 0.3])
def test_strong_coupling_plaquette_gpu(fp64, beta, update):
    p = ml.Params(L=8, Nt=8, beta=beta, seed=200 + int(100 * beta), fp64=fp64, slab=2, n_sub=1, k_between=1,
                  r=(1,), update=update, metro_hits=2, metro_width=2.5)
    with ml.Lattice(p) as lat:
        lat.thermalize(20)
        rec = lat.measure(300)
    plaq = ml.split_record(p, rec)["plaq"]
    m, e = jackknife(plaq.reshape(30, 10).mean(axis=1))
    u = sp.i1(beta) / sp.i0(beta)
    assert abs(m - u) < 3 * e + 10 * u ** 5, (m, e, u)


CHAIN = dict(L=6, Nt=4, beta=0.9, slab=2, n_sub=10, k_between=2, r=(1, 2), rf=(2,), probes=((0, 0), (1, 0)),
             comp_mask=0x3F)


@pytest.fixture(scope="module")
def oracle_chain():
    po = oracle.Params(seed=300, **CHAIN)
    th = oracle.hot_start(po)
    c = oracle.thermalize(po, th, 0, 50)
    rec, _ = oracle.measure(po, th, c, 60)
    return oracle.split_record(po, rec)


def _quantities(s):
    return {
        "plaq": s["plaq"],
        "P1": s["P"][:, 0, 0],
        "P2": s["P"][:, 1, 0],
        "naive1": s["naive"][:, 0, 0],
        "W_Ex_Im_0": s["W"][:, 0, 0, 0, 1, 0],
        "W_Ex_Re_0": s["W"][:, 0, 0, 0, 0, 0],
        "W_Bz_Re_1": s["W"][:, 0, 1, 5, 0, 0],
        "vac_Ex_Re": s["vac"][:, 0, 0],
        "vac_By_Re": s["vac"][:, 4, 0],
    }


@pytest.mark.parametrize("fp64", [True, False])
def test_gpu_chain_agrees_with_oracle_chain(oracle_chain, fp64):
    pm = ml.Params(seed=301, fp64=fp64, **CHAIN)
    with ml.Lattice(pm) as lat:
        lat.thermalize(50)
        rec = lat.measure(240)
    g = _quantities(ml.split_record(pm, rec))
    o = _quantities(oracle_chain)
    for key in g:
        mg, eg = jackknife(ml_bins(g[key]))
        mo, eo = jackknife(ml_bins(o[key]))
        assert abs(mg - mo) < 3 * np.hypot(eg, eo) + 1e-12, (key, mg, eg, mo, eo)


def ml_bins(x, nbins=20):
    n = (len(x) // nbins) * nbins
    return x[:n].reshape(nbins, -1).mean(axis=1)


def test_multilevel_matches_naive_small_workload():
    w = workloads.SMALL_FP64
    pm = ml.Params.from_workload(w, n_sub=20, k_between=2)
    with ml.Lattice(pm) as lat:
        lat.thermalize(w.n_therm)
        rec = lat.measure(150)
    s = ml.split_record(pm, rec)
    for a in range(2):  # r = 1, 2
        m1, e1 = jackknife(ml_bins(s["P"][:, a, 0]))
        mn, en = jackknife(ml_bins(s["naive"][:, a, 0]))
        assert abs(m1 - mn) < 3 * np.hypot(e1, en), (a, m1, e1, mn, en)
        assert e1 < en
    # charge conjugation: Im P+P vanishes
    for a in range(4):
        mi, ei = jackknife(ml_bins(s["P"][:, a, 1]))
        assert abs(mi) < 4 * ei + 1e-15


@pytest.mark.parametrize("fp64", [True, False])
def test_multihit_unbiased_and_reduces_the_error_gpu(fp64):
    """Section II.C's multihit on the same chain as the plain estimator: the
    paired differences of P(r >= 2) average to zero, and the multihit error
    is smaller."""
    base = dict(L=8, Nt=8, beta=1.0, seed=77, fp64=fp64, slab=2, n_sub=20, k_between=2, r=(2, 3, 4))
    s = {}
    for mh in (0, 1):
        p = ml.Params(multihit=mh, **base)
        with ml.Lattice(p) as lat:
            lat.thermalize(40)
            s[mh] = ml.split_record(p, lat.measure(100))["P"][:, :, 0]
    for a in range(3):
        md, ed = jackknife(ml_bins(s[1][:, a] - s[0][:, a]))
        assert abs(md) < 3 * ed, (a, md, ed)
        _, e0 = jackknife(ml_bins(s[0][:, a]))
        _, e1 = jackknife(ml_bins(s[1][:, a]))
        assert e1 < e0, (a, e1, e0)


@pytest.mark.parametrize("fp64", [True, False])
def test_beta_zero_means_vanish_gpu(fp64):
    pm = ml.Params(L=6, Nt=4, beta=0.0, seed=17, fp64=fp64, slab=2, n_sub=4, k_between=1, r=(1, 2), rf=(1, 2),
                   probes=((0, 0), (1, 0)), comp_mask=0x3F)
    with ml.Lattice(pm) as lat:
        rec = lat.measure(60)
    s = ml.split_record(pm, rec)
    for key in ("P", "W", "vac"):
        arr = s[key].reshape(60, -1)
        m, e = jackknife(arr)
        assert np.all(np.abs(m) < 4.5 * e + 1e-15), key
    m, e = jackknife(s["plaq"])
    assert abs(m) < 4 * e


def test_gauge_covariance_gpu_sweep():
    L, Nt = 6, 4
    pm = ml.Params(L=L, Nt=Nt, beta=0.95, seed=31, n_or=0)
    po = oracle.Params(L=L, Nt=Nt, beta=0.95, seed=31, n_or=0)
    th = oracle.hot_start(po)
    lam = workloads.random_gauge(L, Nt, seed=8)
    i = np.arange(po.V)
    x, y, z, t = i % L, (i // L) % L, (i // L ** 2) % L, i // L ** 3

    def fwd(mu):
        c = [t.copy(), x.copy(), y.copy(), z.copy()]
        ext = [Nt, L, L, L]
        c[mu] = (c[mu] + 1) % ext[mu]
        return c[1] + L * (c[2] + L * (c[3] + L * c[0]))

    def gauge(a):
        return np.stack([(a[mu] + lam - lam[fwd(mu)] + np.pi) % TWO_PI - np.pi for mu in range(4)])

    with ml.Lattice(pm) as lat:
        lat.set_angles(th)
        lat.compound_sweeps(1)
        a = lat.get_angles()
        lat.set_angles(gauge(th))
        lat.sweep = 0
        lat.compound_sweeps(1)
        b = lat.get_angles()
    d = np.abs((b - gauge(a) + np.pi) % TWO_PI - np.pi)
    assert d.max() < 1e-10


def test_metropolis_and_heatbath_sample_the_same_ensemble():
    """FP32 chains of 24 lattices (12 per update) at beta = 0.95 on the
    6^3 x 4 multilevel workload: plaquette and P(1) means agree between the
    heatbath and the Metropolis chains within 4 combined standard errors."""
    base = dict(L=6, Nt=4, beta=0.95, fp64=False, slab=2, n_sub=5, k_between=2, r=(1, 2))
    out = {}
    for update in (ml.ML_UPDATE_HEATBATH, ml.ML_UPDATE_METROPOLIS):
        ps = [ml.Params(seed=700 + 31 * i + update, update=update, metro_hits=4, metro_width=1.5, **base)
              for i in range(12)]
        with ml.Batch(ps) as b:
            b.thermalize(100)
            recs = b.measure(20)
        per = [ml.split_record(p, r) for p, r in zip(ps, recs)]
        out[update] = {"plaq": np.array([s["plaq"].mean() for s in per]),
                       "P1": np.array([s["P"][:, 0, 0].mean() for s in per])}
    for key in ("plaq", "P1"):
        a, b = out[0][key], out[1][key]
        ea, eb = a.std(ddof=1) / np.sqrt(a.size), b.std(ddof=1) / np.sqrt(b.size)
        assert abs(a.mean() - b.mean()) < 4 * np.hypot(ea, eb), (key, a.mean(), ea, b.mean(), eb)
