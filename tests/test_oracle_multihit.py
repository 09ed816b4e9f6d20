"""Pins of the oracle's analytic multihit (Section II.C).

* I0, I1 power series against scipy's modified Bessel functions.
* The multihit mean of one temporal link against direct quadrature of the
  conditional law exp(beta k cos(theta + alpha)) (no Bessel functions).
* The same mean against heatbath resampling of that link with the rest of
  the lattice fixed, and the two-line product conj(U(x)) U(x + r) against
  resampling both links (they share no plaquette).
* The n2 = 1 record: P(r >= 2) is the site mean of conj(M(x)) M(x + r) with
  M(x) the time product of the multihit means; P(1), the field records and
  the chain itself are those of the plain estimator.
* Unbiasedness and variance reduction: multihit and plain multilevel P(r)
  agree statistically, the multihit error is smaller.
"""

import numpy as np
import pytest
import scipy.special as sp

import oracle
from paper_1309_3859_b300 import workloads
from paper_1309_3859_b300.stats import jackknife


def _coords(L, Nt):
    i = np.arange(L ** 3 * Nt)
    return i // L ** 3, i % L, (i // L) % L, (i // L ** 2) % L


@pytest.mark.parametrize("x", [0.0, 1e-6, 0.3, 1.0, 2.5, 6.0, 17.0, 60.0, 300.0])
def test_bessel_series_against_scipy(x):
    assert abs(oracle.bessel_i0(x) - sp.i0(x)) <= 1e-14 * sp.i0(x)
    assert abs(oracle.bessel_i1(x) - sp.i1(x)) <= 1e-14 * max(sp.i1(x), 1e-300)


def test_multihit_link_against_quadrature():
    """<e^{i theta}> = int e^{i theta} e^{beta k cos(theta + alpha)} / int e^{...};
    the trapezoid rule on a periodic analytic integrand converges exponentially."""
    L, Nt = 4, 4
    p = oracle.Params(L=L, Nt=Nt, beta=1.05)
    th = workloads.random_angles(L, Nt, seed=17)
    grid = np.linspace(0, 2 * np.pi, 4096, endpoint=False)
    for i in range(0, p.V, 7):
        W = oracle.staple(p, th, 0, i)
        w = np.exp(p.beta * np.abs(W) * np.cos(grid + np.angle(W)))
        expect = (np.exp(1j * grid) * w).sum() / w.sum()
        got = oracle.multihit_link(p, th, i)
        assert abs(got - expect) < 1e-13, (i, got, expect)


def test_multihit_link_against_heatbath_resampling():
    """Averaging e^{i theta} over heatbath draws of one checkerboard class of
    temporal links (all other links fixed) converges to the multihit mean;
    for r even, x and x + r are in the same class and the two-line product
    converges to conj(<U>(x)) <U>(x + r)."""
    L, Nt, r = 4, 4, 2
    p = oracle.Params(L=L, Nt=Nt, beta=0.9, seed=8)
    th0 = workloads.random_angles(L, Nt, seed=9)
    t, x, y, z = _coords(L, Nt)
    idx = np.flatnonzero((t + x + y + z) % 2 == 0)
    partner = idx - x[idx] + (x[idx] + r) % L
    mh = np.array([oracle.multihit_link(p, th0, int(i)) for i in range(p.V)])
    n = 3000
    s1 = np.zeros(len(idx), complex)
    s2 = np.zeros(len(idx), complex)
    q1 = np.zeros(len(idx))
    q2 = np.zeros(len(idx))
    for k in range(n):
        th = th0.copy()
        oracle.update_pass(p, th, 0, 0, 0, k + 1, 0)
        u = np.exp(1j * th[0])
        a = u[idx]
        b = np.conj(u[idx]) * u[partner]
        s1 += a
        s2 += b
        q1 += np.abs(a) ** 2
        q2 += np.abs(b) ** 2
    for s, q, expect in ((s1, q1, mh[idx]), (s2, q2, np.conj(mh[idx]) * mh[partner])):
        m = s / n
        se = np.sqrt(np.maximum(q / n - np.abs(m) ** 2, 1e-12) / n)
        z = np.abs(m - expect) / se
        assert z.max() < 6, z.max()
        assert 0.5 < np.mean(z ** 2) < 3.0  # |complex residual|^2 / se^2 averages 1 for 2 dof / 2


def test_single_sub_update_identity_multihit():
    kw = dict(L=6, Nt=4, beta=0.8, seed=3, slab=2, n_sub=1, k_between=1, r=(1, 2, 3, 5), rf=(2, 3),
              probes=((0, 0), (1, 0)), comp_mask=0x3F)
    pm = oracle.Params(multihit=1, **kw)
    pp = oracle.Params(multihit=0, **kw)
    th_m = oracle.hot_start(pm)
    th_p = th_m.copy()
    rec_m, c_m = oracle.measure(pm, th_m, 0, 1)
    rec_p, c_p = oracle.measure(pp, th_p, 0, 1)
    assert c_m == c_p and np.array_equal(th_m, th_p)  # the chain is untouched
    sm, sp_ = oracle.split_record(pm, rec_m[0]), oracle.split_record(pp, rec_p[0])
    L, Nt = pm.L, pm.Nt
    mh = np.array([oracle.multihit_link(pm, th_m, i) for i in range(pm.V)]).reshape(Nt, L, L, L)
    M = mh.prod(axis=0)  # [z, y, x]
    for a, r in enumerate(pm.r):
        if 2 <= r <= L - 2:
            expect = (np.conj(M) * np.roll(M, -r, axis=2)).mean()
            got = sm["P"][a, 0] + 1j * sm["P"][a, 1]
            assert abs(got - expect) < 1e-14, (r, got, expect)
            assert abs(got - (sp_["P"][a, 0] + 1j * sp_["P"][a, 1])) > 1e-6
        else:  # adjacent lines (r = 1, r = L - 1) keep the plain estimator
            assert np.array_equal(sm["P"][a], sp_["P"][a])
    for key in ("Pf", "W", "vac", "naive"):
        assert np.array_equal(sm[key], sp_[key]), key


def test_multihit_unbiased_and_reduces_the_error():
    base = dict(L=6, Nt=4, beta=0.9, slab=2, n_sub=8, k_between=2, r=(2, 3), threads=4)
    pm = oracle.Params(seed=41, multihit=1, **base)
    pp = oracle.Params(seed=41, multihit=0, **base)
    th = oracle.hot_start(pm)
    c = oracle.thermalize(pm, th, 0, 30)
    th2 = th.copy()
    rec_m, _ = oracle.measure(pm, th, c, 40)
    rec_p, _ = oracle.measure(pp, th2, c, 40)
    sm, sp_ = oracle.split_record(pm, rec_m), oracle.split_record(pp, rec_p)
    for a in range(2):
        mm, em = jackknife(sm["P"][:, a, 0])
        mp, ep = jackknife(sp_["P"][:, a, 0])
        mn, en = jackknife(sp_["naive"][:, a, 0])
        assert abs(mm - mp) < 3 * np.hypot(em, ep), (a, mm, em, mp, ep)
        assert abs(mm - mn) < 3 * np.hypot(em, en), (a, mm, em, mn, en)
        assert em < ep, (a, em, ep)


@pytest.mark.parametrize("bad", [dict(multihit=2), dict(multihit=1, beta=150.0)])
def test_multihit_validation(bad):
    kw = dict(L=4, Nt=4, beta=1.0)
    kw.update(bad)
    assert oracle.validate(oracle.Params(**kw)) != 0
