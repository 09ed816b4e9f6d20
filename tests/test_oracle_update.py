"""Pins of the oracle's action, link updates and sweep structure.

* Plaquette field, mean plaquette and action on uniform-flux configurations
  whose plaquettes are known in closed form (Section II, Wilson action).
* The staple sum against finite differences of the total action.
* Overrelaxation: local action unchanged, involution, total action unchanged.
* Heatbath: theta + alpha follows the von Mises law of kappa = beta k, tested
  by the probability-integral transform through scipy's von Mises CDF.
* Metropolis (the paper's update, Section II): the conditional law is
  stationary under a Metropolis pass (links drawn from it by the heatbath stay
  distributed by it), the pass moves links at a sane rate, and a Metropolis
  chain reaches the strong-coupling plaquette.
* Slab freezing and checkerboard parity of the passes.
* The whole chain against the strong-coupling plaquette I1(beta)/I0(beta).
* Gauge covariance of the chain and invariance of the observables.
* beta = 0: uniform links, zero mean plaquette.
"""

import numpy as np
import pytest
import scipy.special as sp
import scipy.stats as st

import oracle
from paper_1309_3859_b300 import workloads
from paper_1309_3859_b300.stats import jackknife

TWO_PI = 2 * np.pi


def wrapd(a):
    """distance on the circle"""
    return np.abs((a + np.pi) % TWO_PI - np.pi)


def coords(L, Nt):
    i = np.arange(L ** 3 * Nt)
    x = i % L
    y = (i // L) % L
    z = (i // L ** 2) % L
    t = i // L ** 3
    return t, x, y, z


def site_shift(L, Nt, mu, sign):
    """index of i + sign*mu-hat for every site i"""
    t, x, y, z = coords(L, Nt)
    c = [t, x, y, z]
    ext = [Nt, L, L, L]
    c = [a.copy() for a in c]
    c[mu] = (c[mu] + sign) % ext[mu]
    return c[1] + L * (c[2] + L * (c[3] + L * c[0]))


# --------------------------------------------------------------------------- closed forms
@pytest.mark.parametrize("comp", range(6))
def test_plaquette_field_uniform_flux(comp):
    L, Nt = 4, 6
    p = oracle.Params(L=L, Nt=Nt, beta=1.3)
    t, x, y, z = coords(L, Nt)
    th = np.zeros((4, p.V))
    b = TWO_PI / L  # b L = 2 pi makes the flux uniform across the periodic wrap
    bt = TWO_PI / Nt
    # (direction that carries the gradient, coordinate it grows along, step)
    recipe = {0: (1, t, bt), 1: (2, t, bt), 2: (3, t, bt), 3: (3, y, b), 4: (1, z, b), 5: (2, x, b)}
    mu, coord, step = recipe[comp]
    th[mu] = step * coord
    th = (th + np.pi) % TWO_PI - np.pi
    f = oracle.plaquette_field(p, th)
    for c in range(6):
        if c == comp:
            assert np.allclose(f[c, 0], np.cos(step), atol=1e-14)
            assert np.allclose(f[c, 1], np.sin(step), atol=1e-14)
        else:
            assert np.allclose(f[c, 0], 1.0, atol=1e-14)
            assert np.allclose(f[c, 1], 0.0, atol=1e-14)
    pm = oracle.plaquette_mean(p, th)
    assert abs(pm - (5 + np.cos(step)) / 6) < 1e-14
    assert abs(oracle.action(p, th) - p.beta * p.V * (1 - np.cos(step))) < 1e-10


def test_staple_against_action_differences():
    L, Nt = 4, 4
    p = oracle.Params(L=L, Nt=Nt, beta=0.7)
    th0 = workloads.random_angles(L, Nt, seed=3)
    rng = np.random.default_rng(4)
    for _ in range(12):
        mu = int(rng.integers(4))
        i = int(rng.integers(p.V))
        w = oracle.staple(p, th0, mu, i)
        S = {}
        for a in (0.0, np.pi, np.pi / 2, -np.pi / 2):
            th = th0.copy()
            th[mu, i] = a
            S[a] = oracle.action(p, th)
        # S(a) = C - beta (Re W cos a - Im W sin a)
        wr = (S[np.pi] - S[0.0]) / (2 * p.beta)
        wi = (S[np.pi / 2] - S[-np.pi / 2]) / (2 * p.beta)
        assert abs(wr - w.real) < 1e-10 and abs(wi - w.imag) < 1e-10


# --------------------------------------------------------------------------- overrelaxation
def test_overrelaxation_invariants():
    L, Nt = 4, 4
    p = oracle.Params(L=L, Nt=Nt, beta=0.9)
    th0 = workloads.random_angles(L, Nt, seed=5)
    t, x, y, z = coords(L, Nt)
    par = (t + x + y + z) % 2
    S0 = oracle.action(p, th0)
    for mu in range(4):
        for parity in range(2):
            th = th0.copy()
            oracle.update_pass(p, th, mu, parity, 0, 1, 1)
            # only links (mu, parity) move
            moved = wrapd(th - th0) > 0
            assert not moved[[m for m in range(4) if m != mu]].any()
            assert not moved[mu][par != parity].any()
            assert moved[mu][par == parity].all()
            # local action unchanged: cos(theta' + alpha) = cos(theta + alpha)
            for i in np.flatnonzero(par == parity)[:40]:
                w = oracle.staple(p, th0, mu, int(i))
                a = np.angle(w)
                assert abs(np.cos(th[mu, i] + a) - np.cos(th0[mu, i] + a)) < 1e-13
            # total action unchanged, and the pass is an involution
            assert abs(oracle.action(p, th) - S0) < 1e-11 * abs(S0)
            oracle.update_pass(p, th, mu, parity, 0, 1, 1)
            assert wrapd(th - th0).max() < 1e-13


# --------------------------------------------------------------------------- heatbath
@pytest.mark.parametrize("draws", [0, 1])
def test_heatbath_conditional_law(draws):
    L, Nt = 4, 4
    p = oracle.Params(L=L, Nt=Nt, beta=1.1, draws=draws, seed=21)
    th0 = workloads.random_angles(L, Nt, seed=6)
    t, x, y, z = coords(L, Nt)
    par = (t + x + y + z) % 2
    us = []
    for mu, parity in ((0, 0), (2, 1)):
        idx = np.flatnonzero(par == parity)
        W = np.array([oracle.staple(p, th0, mu, int(i)) for i in idx])
        kappa = p.beta * np.abs(W)
        alpha = np.angle(W)
        for n in range(1, 161):
            th = th0.copy()
            oracle.update_pass(p, th, mu, parity, 0, n, 0)
            psi = (th[mu, idx] + alpha + np.pi) % TWO_PI - np.pi
            us.append(st.vonmises.cdf(psi, kappa))
            untouched = np.ones(p.V, bool)
            untouched[idx] = False
            assert np.array_equal(th[mu, untouched], th0[mu, untouched])
    u = np.concatenate(us)
    counts, _ = np.histogram(u, bins=40, range=(0, 1))
    assert st.chisquare(counts).pvalue > 1e-4


# --------------------------------------------------------------------------- Metropolis
@pytest.mark.parametrize("draws", [0, 1])
def test_metropolis_keeps_the_conditional_law(draws):
    """Links drawn from their conditional law exp(beta k cos(theta + alpha))
    (by a heatbath pass) still follow it after a Metropolis pass of the same
    links with fresh random numbers: the law is stationary.  An inverted or
    mis-scaled acceptance ratio shifts the distribution and fails."""
    L, Nt = 4, 4
    p = oracle.Params(L=L, Nt=Nt, beta=1.3, draws=draws, seed=31, update=1, metro_hits=3, metro_width=1.7)
    th0 = workloads.random_angles(L, Nt, seed=8)
    t, x, y, z = coords(L, Nt)
    par = (t + x + y + z) % 2
    us, moved = [], []
    for mu, parity in ((1, 0), (0, 1)):
        idx = np.flatnonzero(par == parity)
        W = np.array([oracle.staple(p, th0, mu, int(i)) for i in idx])
        kappa, alpha = p.beta * np.abs(W), np.angle(W)
        for n in range(1, 201):
            th = th0.copy()
            oracle.update_pass(p, th, mu, parity, 0, n, 0)           # exact draw
            before = th[mu, idx].copy()
            oracle.update_pass(p, th, mu, parity, 0, 100000 + n, 2)  # Metropolis
            psi = (th[mu, idx] + alpha + np.pi) % TWO_PI - np.pi
            us.append(st.vonmises.cdf(psi, kappa))
            moved.append(wrapd(th[mu, idx] - before) > 0)
    u = np.concatenate(us)
    counts, _ = np.histogram(u, bins=40, range=(0, 1))
    assert st.chisquare(counts).pvalue > 1e-4
    rate = np.concatenate(moved).mean()
    assert 0.3 < rate < 0.99, rate


def test_metropolis_pass_matches_its_definition():
    """One Metropolis hit per link, recomputed in numpy from the Philox
    draws: proposal theta + w (2 u1 - 1), accepted when u2 < exp(beta k
    (cos(theta' + alpha) - cos(theta + alpha)))."""
    L, Nt = 4, 4
    p = oracle.Params(L=L, Nt=Nt, beta=0.9, draws=0, seed=41, update=1, metro_hits=1, metro_width=0.8)
    th0 = workloads.random_angles(L, Nt, seed=12)
    t, x, y, z = coords(L, Nt)
    par = (t + x + y + z) % 2
    mu, parity, n = 2, 0, 7
    th = th0.copy()
    oracle.update_pass(p, th, mu, parity, 0, n, 2)
    key = np.array([p.seed & 0xFFFFFFFF, p.seed >> 32], dtype=np.uint32)
    for i in np.flatnonzero(par == parity)[:40]:
        W = oracle.staple(p, th0, mu, int(i))
        k, alpha = abs(W), np.angle(W)
        o = oracle.philox(np.array([[i, mu, n, 0]], dtype=np.uint32), key[None, :])[0]
        u1 = oracle.uniform52(int(o[0]), int(o[1]))
        u2 = oracle.uniform52(int(o[2]), int(o[3]))
        prop = (th0[mu, i] + 0.8 * (2 * u1 - 1) + np.pi) % TWO_PI - np.pi
        ds = 0.9 * k * (np.cos(prop + alpha) - np.cos(th0[mu, i] + alpha))
        want = prop if (ds >= 0 or u2 < np.exp(ds)) else th0[mu, i]
        assert wrapd(th[mu, i] - want) < 1e-13, i


# --------------------------------------------------------------------------- sweep structure
@pytest.mark.parametrize("d", [2, 4])
def test_slab_mask_freezes_boundary_spatial_links(d):
    L, Nt = 4, 8
    p = oracle.Params(L=L, Nt=Nt, beta=0.95, seed=9)
    th0 = oracle.hot_start(p)
    th = th0.copy()
    oracle.compound_sweep(p, th, 0, slab_d=d)
    t, _, _, _ = coords(L, Nt)
    moved = wrapd(th - th0) > 0
    assert moved[0].all()  # temporal links always update
    for mu in (1, 2, 3):
        assert not moved[mu][t % d == 0].any()
        assert moved[mu][t % d != 0].all()


def test_hot_start_uniform():
    p = oracle.Params(L=8, Nt=4, beta=1.0, seed=77)
    th = oracle.hot_start(p).ravel()
    assert th.min() >= -np.pi and th.max() < np.pi
    counts, _ = np.histogram(th, bins=32, range=(-np.pi, np.pi))
    assert st.chisquare(counts).pvalue > 1e-4


# --------------------------------------------------------------------------- whole chain
@pytest.mark.parametrize("update", [0, 1])
@pytest.mark.parametrize("beta", [0.05, 0.1, 0.2, 0.3])
def test_strong_coupling_plaquette(beta, update):
    """<cos theta_p> = u + O(u^5), u = I1(beta)/I0(beta), for heatbath and
    Metropolis chains."""
    p = oracle.Params(L=4, Nt=4, beta=beta, seed=100 + int(beta * 100), threads=4, update=update, metro_hits=2,
                      metro_width=2.5)
    th = oracle.hot_start(p)
    c = oracle.thermalize(p, th, 0, 20)
    vals = []
    for _ in range(300):
        c = oracle.compound_sweep(p, th, c)
        vals.append(oracle.plaquette_mean(p, th))
    m, e = jackknife(np.array(vals).reshape(30, 10).mean(axis=1))
    u = sp.i1(beta) / sp.i0(beta)
    assert abs(m - u) < 3 * e + 10 * u ** 5, (beta, m, e, u)


def _gauge(th, lam, L, Nt):
    out = np.empty_like(th)
    for mu in range(4):
        out[mu] = (th[mu] + lam - lam[site_shift(L, Nt, mu, +1)] + np.pi) % TWO_PI - np.pi
    return out


def test_gauge_covariance_one_heatbath_sweep():
    """At beta near the transition one heatbath sweep is covariant to rounding.

    (Longer chains there amplify rounding by about 100x per sweep, so the
    multi-sweep check below runs in the ordered phase.)"""
    L, Nt = 4, 4
    p = oracle.Params(L=L, Nt=Nt, beta=0.95, seed=31, n_or=0)
    th = oracle.hot_start(p)
    lam = workloads.random_gauge(L, Nt, seed=8)
    a, b = th.copy(), _gauge(th, lam, L, Nt)
    oracle.compound_sweep(p, a, 0)
    oracle.compound_sweep(p, b, 0)
    ga = _gauge(a, lam, L, Nt)
    assert wrapd(b - ga).max() < 1e-10
    assert abs(oracle.plaquette_mean(p, a) - oracle.plaquette_mean(p, b)) < 1e-12
    for r in (1, 2, 3):
        assert abs(oracle.naive_correlator(p, a, r) - oracle.naive_correlator(p, b, r)) < 1e-12


def test_gauge_invariance_of_the_measurement():
    L, Nt = 4, 8
    p = oracle.Params(L=L, Nt=Nt, beta=2.5, seed=31, slab=2, n_sub=3, outer_slab=4, n_sub_outer=2, k_between=1,
                      r=(1, 2), rf=(1, 2, 3), probes=((0, 0), (1, 0), (-1, 1)), comp_mask=0x3F)
    th = np.zeros((4, p.V))
    c = oracle.thermalize(p, th, 0, 10)
    lam = workloads.random_gauge(L, Nt, seed=8)
    a, b = th.copy(), _gauge(th, lam, L, Nt)
    ra, ca = oracle.measure(p, a, c, 2)
    rb, cb = oracle.measure(p, b, c, 2)
    assert ca == cb
    assert wrapd(b - _gauge(a, lam, L, Nt)).max() < 1e-9
    assert np.abs(ra - rb).max() < 1e-9
    assert np.abs(oracle.plaquette_field(p, a) - oracle.plaquette_field(p, b)).max() < 1e-9


def test_beta_zero_links_uniform():
    p = oracle.Params(L=4, Nt=4, beta=0.0, seed=41)
    th = oracle.hot_start(p)
    c = 0
    vals, ims = [], []
    for _ in range(100):
        c = oracle.compound_sweep(p, th, c)
        vals.append(oracle.plaquette_mean(p, th))
        ims.append(oracle.plaquette_field(p, th)[:, 1].mean())
    sigma = np.sqrt(0.5 / (6 * p.V * len(vals)))
    assert abs(np.mean(vals)) < 4 * sigma
    assert abs(np.mean(ims)) < 4 * sigma
    counts, _ = np.histogram(th.ravel(), bins=16, range=(-np.pi, np.pi))
    assert st.chisquare(counts).pvalue > 1e-4
