"""Pins of the oracle's multilevel estimators (Section II.C, Algorithm 1).

* n2 = 1 identity: the product of the slab two-link operators of one
  configuration is P(x)^* P(x + r xhat), and the field-insertion sum is
  P^* P times the time sum of the plaquette at the probe (one and two levels).
* Vacuum sums equal the plaquette means of the sub-update configurations.
* Strong coupling: multilevel P(r) against u^(r Nt), u = I1(beta)/I0(beta).
* Unbiasedness: multilevel and naive P(r) agree; one and two levels agree.
* Symmetries: <P> = 0 (U(1) centre symmetry) and Im <P^* P> = 0 (charge
  conjugation).
"""

import numpy as np
import pytest
import scipy.special as sp

import oracle
from ml_identity import _identity_expectation
from paper_1309_3859_b300.stats import jackknife


@pytest.mark.parametrize("two_level", [False, True])
def test_single_sub_update_identity(two_level):
    kw = dict(outer_slab=4, n_sub_outer=1) if two_level else {}
    p = oracle.Params(L=4, Nt=8, beta=0.8, seed=3, slab=2, n_sub=1, k_between=1, r=(1, 2, 3),
                      rf=(1, 2, 3), probes=((0, 0), (1, 0), (0, 1), (-1, 2)), comp_mask=0x3F, **kw)
    th = oracle.hot_start(p)
    rec, _ = oracle.measure(p, th, 0, 1)
    s = oracle.split_record(p, rec[0])
    Pexp, Wexp = _identity_expectation(p, th)
    assert np.abs(s["P"][:, 0] + 1j * s["P"][:, 1] - Pexp).max() < 1e-13
    Pf = s["Pf"][:, 0] + 1j * s["Pf"][:, 1]
    assert np.abs(Pf - Pexp[[p.r.index(r) for r in p.rf]]).max() < 1e-13
    Wgot = s["W"][..., 0] + 1j * s["W"][..., 1]
    assert np.abs(Wgot - Wexp).max() < 1e-13
    # vacuum sums: one configuration, site means of Re / Im P_c
    f = oracle.plaquette_field(p, th)
    assert np.abs(s["vac"] - f.mean(axis=2)).max() < 1e-14


def test_component_mask_zeroes_unselected():
    p = oracle.Params(L=4, Nt=4, beta=0.8, seed=3, slab=2, n_sub=2, r=(1,), rf=(2,), probes=((0, 0),),
                      comp_mask=0b001001)
    th = oracle.hot_start(p)
    rec, _ = oracle.measure(p, th, 0, 1)
    s = oracle.split_record(p, rec[0])
    for c in range(6):
        sel = c in (0, 3)
        assert (np.abs(s["W"][:, :, c]).max() > 0) == sel
        assert (np.abs(s["vac"][c]).max() > 0) == sel


def test_vacuum_is_mean_plaquette_of_sub_updates():
    p = oracle.Params(L=4, Nt=4, beta=0.9, seed=5, slab=2, n_sub=3, k_between=0, r=(1,), comp_mask=0x3F)
    th = oracle.hot_start(p)
    a = th.copy()
    c = 0
    plaqs = []
    for _ in range(3):
        c = oracle.compound_sweep(p, a, c, slab_d=2)
        plaqs.append(oracle.plaquette_mean(p, a))
    rec, c2 = oracle.measure(p, th, 0, 1)
    s = oracle.split_record(p, rec[0])
    assert c2 == c
    assert np.abs(th - a).max() == 0.0
    assert abs(s["vac"][:, 0].mean() - np.mean(plaqs)) < 1e-14


def test_multilevel_strong_coupling_correlator():
    """P(r=1) = u^(r Nt) (1 + O(A u^4)) at beta = 0.3 (A = r Nt plaquettes)."""
    beta = 0.3
    p = oracle.Params(L=6, Nt=4, beta=beta, seed=12, slab=2, n_sub=200, k_between=2, r=(1,))
    th = oracle.hot_start(p)
    c = oracle.thermalize(p, th, 0, 20)
    rec, _ = oracle.measure(p, th, c, 20)
    P = oracle.split_record(p, rec)["P"][:, 0, 0]
    m, e = jackknife(P)
    u = sp.i1(beta) / sp.i0(beta)
    expect = u ** 4
    assert abs(m - expect) < 3 * e + 0.05 * expect, (m, e, expect)
    assert e < 0.2 * expect  # the multilevel estimate resolves the signal


def test_multilevel_agrees_with_naive_and_two_level():
    base = dict(L=4, Nt=8, beta=0.7, slab=2, k_between=2, r=(1, 2), threads=4)
    p1 = oracle.Params(seed=21, n_sub=12, **base)
    th = oracle.hot_start(p1)
    c = oracle.thermalize(p1, th, 0, 30)
    rec1, c = oracle.measure(p1, th, c, 40)
    s1 = oracle.split_record(p1, rec1)
    p2 = oracle.Params(seed=22, n_sub=6, outer_slab=4, n_sub_outer=3, **base)
    rec2, _ = oracle.measure(p2, th, c, 25)
    s2 = oracle.split_record(p2, rec2)
    for a in range(2):
        m1, e1 = jackknife(s1["P"][:, a, 0])
        mn, en = jackknife(np.concatenate([s1["naive"][:, a, 0], s2["naive"][:, a, 0]]))
        m2, e2 = jackknife(s2["P"][:, a, 0])
        assert abs(m1 - mn) < 3 * np.hypot(e1, en), (a, m1, e1, mn, en)
        assert abs(m2 - mn) < 3 * np.hypot(e2, en), (a, m2, e2, mn, en)
        assert abs(m1 - m2) < 3 * np.hypot(e1, e2), (a, m1, e1, m2, e2)
        assert e1 < en  # multilevel reduces the error
        # charge conjugation: the imaginary part vanishes
        mi, ei = jackknife(s1["P"][:, a, 1])
        assert abs(mi) < 4 * ei + 1e-15


def test_polyakov_loop_vanishes():
    p = oracle.Params(L=4, Nt=4, beta=0.9, seed=33)
    th = oracle.hot_start(p)
    c = oracle.thermalize(p, th, 0, 20)
    vals = []
    for _ in range(60):
        c = oracle.compound_sweep(p, th, c)
        vals.append(oracle.polyakov(p, th).mean())
    vals = np.array(vals)
    for part in (vals.real, vals.imag):
        m, e = jackknife(part)
        assert abs(m) < 4 * e


def test_beta_zero_multilevel_means_vanish():
    p = oracle.Params(L=4, Nt=4, beta=0.0, seed=44, slab=2, n_sub=4, k_between=1, r=(1, 2), rf=(1, 2),
                      probes=((0, 0), (1, 0)), comp_mask=0x3F)
    th = oracle.hot_start(p)
    rec, _ = oracle.measure(p, th, 0, 30)
    s = oracle.split_record(p, rec)
    for arr in (s["P"].reshape(30, -1), s["W"].reshape(30, -1), s["vac"].reshape(30, -1)):
        m, e = jackknife(arr)
        assert np.all(np.abs(m) < 4.5 * e + 1e-15)


@pytest.mark.parametrize("bad", [
    dict(L=5), dict(Nt=3), dict(beta=-0.1), dict(slab=3), dict(n_sub=0), dict(outer_slab=3),
    dict(outer_slab=8, n_sub_outer=1, Nt=4), dict(outer_slab=4, n_sub_outer=0), dict(r=(0,)), dict(r=(4,)),
    dict(rf=(5,)), dict(probes=((4, 0),)), dict(probes=((0, -4),)), dict(comp_mask=64), dict(k_between=-1),
])
def test_parameter_validation(bad):
    kw = dict(L=4, Nt=4, beta=1.0, slab=2, n_sub=1, r=(1,), rf=(1,), probes=((0, 0),), comp_mask=1)
    kw.update(bad)
    assert oracle.validate(oracle.Params(**kw)) == -1
    kw2 = dict(L=4, Nt=4, beta=1.0, slab=2, n_sub=1, r=(1,), rf=(1,), probes=((0, 0),), comp_mask=1)
    assert oracle.validate(oracle.Params(**kw2)) == 0
